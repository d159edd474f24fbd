"""Seeded synthetic inputs for the shifted Sternheimer solve (shared by the CUDA path and the oracle)."""
from .generate import (HA_EV, Instance, KPointData, config1, config2, config3, config4, config4_spec, fcc_perturbed, tiny_fcc,
                       ground_state, make_instance)

__all__ = ["HA_EV", "Instance", "KPointData", "config1", "config2", "config3", "config4", "config4_spec", "fcc_perturbed", "tiny_fcc",
           "ground_state", "make_instance"]
