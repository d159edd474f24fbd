// The shifted Lanczos kernel in the ArDF arithmetic policy (one translation unit per policy,
// so the three compile in parallel).
#include "lanczos.cuh"

namespace sgw {

int lanczos_smem_df(const Plan& P, int nshift) { return lanczos_smem_t<ArDF>(P, nshift); }

cudaError_t lanczos_capacity_df(const Plan& P, int nshift, int threads, int* owners) {
    return lanczos_capacity_t<ArDF>(P, nshift, threads, owners);
}

cudaError_t lanczos_launch_df(const Plan& P, const LanczosArgs& a, int owners, int threads, cudaStream_t st) {
    return lanczos_launch_t<ArDF>(P, a, owners, threads, st);
}

cudaError_t lanczos_batch_capacity_df(const Plan& P, int threads, int smem, int* owners) {
    return lanczos_batch_capacity_t<ArDF>(P, threads, smem, owners);
}

cudaError_t lanczos_batch_launch_df(const Plan& P, const BatchItem* items, const int* start, int nitems, int* counter,
                                    int owners, int threads, int smem, cudaStream_t st) {
    return lanczos_batch_launch_t<ArDF>(P, items, start, nitems, counter, owners, threads, smem, st);
}

}  // namespace sgw
