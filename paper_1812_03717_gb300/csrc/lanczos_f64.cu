// The shifted Lanczos kernel in the ArF64 arithmetic policy (one translation unit per policy,
// so the three compile in parallel).
#include "lanczos.cuh"

namespace sgw {

int lanczos_smem_f64(const Plan& P, int nshift) { return lanczos_smem_t<ArF64>(P, nshift); }

cudaError_t lanczos_capacity_f64(const Plan& P, int nshift, int threads, int* owners) {
    return lanczos_capacity_t<ArF64>(P, nshift, threads, owners);
}

cudaError_t lanczos_launch_f64(const Plan& P, const LanczosArgs& a, int owners, int threads, cudaStream_t st) {
    return lanczos_launch_t<ArF64>(P, a, owners, threads, st);
}

cudaError_t lanczos_batch_capacity_f64(const Plan& P, int threads, int smem, int* owners) {
    return lanczos_batch_capacity_t<ArF64>(P, threads, smem, owners);
}

cudaError_t lanczos_batch_launch_f64(const Plan& P, const BatchItem* items, const int* start, int nitems, int* counter,
                                    int owners, int threads, int smem, cudaStream_t st) {
    return lanczos_batch_launch_t<ArF64>(P, items, start, nitems, counter, owners, threads, smem, st);
}

}  // namespace sgw
