// Host-side launchers of the set-up kernels (setup.cu) and the hot kernels (kernels.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sgw_internal.cuh"

namespace sgw {

struct SphereArgs {
    double b[3][3];   // reciprocal lattice rows (bohr^-1)
    double k[3];      // fractional k
    double ecut;      // Ry == bohr^-2
    int M[3];         // Miller bounds
    int cap;          // capacity of the output arrays
};

struct BetaArgs {
    double b[3][3];
    double k[3];
    double inv_sqrt_vol;
    double width[64];
    double tau[64][3];
};
constexpr int kMaxProj = 64;

struct RhsArgs {
    int lo[3];
    int ext[3];
};

cudaError_t launch_sphere(const SphereArgs& a, int* miller, double* kin, int* count, cudaStream_t st);
cudaError_t launch_boxmap(const int* miller, int npw, const int dims[3], int* map, cudaStream_t st);
cudaError_t launch_beta(const BetaArgs& a, int nproj, const int* miller, int npw, double2* beta, cudaStream_t st);
cudaError_t launch_twiddles(const int dims[3], double2* tw, cudaStream_t st);
cudaError_t launch_rhs(const RhsArgs& a, const int* miller_kq, int npw_kq, const int* lut_k, const double2* psi_k,
                       int npw_k, const int* gp, int n_v, int n_pert, double2* rhs, cudaStream_t st);
cudaError_t launch_gram(const double2* psi, int nocc, int npw, double2* S, cudaStream_t st);
cudaError_t launch_to_dd(const double* src, size_t n, float2* dst, cudaStream_t st);

// --- hot path (kernels.cu)

struct SolveArgs {
    int nrhs, nshift, ell, max_mv;
    const double2* rhs;       // [nrhs][npw]
    const double* e_ref;      // [nrhs]
    const double* sig;        // [nshift]  z_seed - z_j (real: omega_seed - omega_j)
    double omega_seed, eta, tol;
    double2* x;               // [nrhs][nshift][npw]   (the caller's dpsi)
    double2* uw;              // [grid][nshift][npw]   per-CTA shift directions
    double2* seedw;           // [grid][2 ell + 3][npw] per-CTA seed vectors
    int* counter;             // work queue (zeroed by the launcher)
    int* out_mv;              // [nrhs][nshift]
    double* out_res;          // [nrhs][nshift]
    int* out_status;          // [nrhs][nshift]
    const double* pre = nullptr;   // [nrhs][npw] right diagonal preconditioner (nshift == 1 only)
    double2* pscr = nullptr;       // [grid][2][npw] scratch for the preconditioned operator
};

struct PrecondArgs {
    int n;                         // items (single-shift systems)
    int mode;                      // SGW_PRECOND_PLAIN / _JACOBI / _LEARNED
    const double2* rhs;            // [n][npw]
    const double* e_ref;           // [n]
    const double* omega;           // [n]
    const double* delta;           // [n] Jacobi floors (JACOBI)
    double eta;
    double half_ecut;              // E_cut / 2 (Ha)
    double v_mean;                 // <V_loc> (Ha)
    const __nv_bfloat16* mlp;      // packed perceptron weights (LEARNED)
    double* d;                     // [n][npw] out
};
cudaError_t launch_precond(const Plan& P, const PrecondArgs& a, cudaStream_t st);

struct TrainRowsArgs {
    int n;
    const double2* rhs;            // [n][npw]
    const double* e_ref;           // [n]
    const double* omega;           // [n]
    const double* delta;           // [n] best Jacobi floor of each pair (<= 0: plain was best)
    double eta, half_ecut, v_mean;
    float* feats;                  // [n * npw][4]
    float* targets;                // [n * npw]
};
cudaError_t launch_training_rows(const Plan& P, const TrainRowsArgs& a, cudaStream_t st);
const __nv_bfloat16* mlp_weights(const sgw_mlp* m);

struct LanczosArgs {
    int nrhs, nshift, maxk;
    const double2* rhs;       // [nrhs][npw]
    const double* e_ref;      // [nrhs]
    const double* omega;      // [nshift]
    double eta, tol;
    double2* x;               // [nrhs][nshift][npw]
    double2* basis;           // [grid][maxk + 1][npw]
    double* ab;               // [grid][2][maxk + 1]
    double2* ysc;             // [grid][2][maxk][nshift]
    int* counter;
    int* out_mv;              // [nrhs][nshift]  Lanczos steps when the pair converged
    double* out_res;          // [nrhs][nshift]
    int* out_status;          // [nrhs][nshift]
    // Im z_rj: eta_r[r] when given, else eta_s[j] when given, else eta (any sign but 0)
    const double* eta_s = nullptr;   // [nshift]
    const double* eta_r = nullptr;   // [nrhs]
    double cert_tol = 0.0;           // > 0: shifts also stop only once |r| / (|Im z| |x|) <= cert_tol
    size_t vstride = 0;              // basis elements per owner (0: (maxk + 1) npw)
    size_t ystride = 0;              // y / l coefficients per CTA (0: 2 maxk nshift)
};

// One system of a packed multi-system launch.
struct BatchItem {
    Plan plan;
    LanczosArgs args;
};

// Bytes per complex value of a precision's arithmetic policy.
inline int prec_bytes(int precision) { return precision == SGW_PREC_FP32 ? 8 : 16; }

// Launch plumbing shared by the kernels that own one vector per CTA or per cluster.
int optin_smem();
cudaError_t allow_max_smem(const void* kernel);
Plan tuned_plan(const Plan& P, int extra, int es);
cudaError_t owner_capacity(const void* kernel, const Plan& P, int threads, int smem, int* owners);
cudaError_t launch_owned(const void* kernel, const Plan& P, int owners, int threads, int smem, cudaStream_t st,
                         void** args);

// Multishift Lanczos in the policy of `precision`; owners = right-hand sides in flight (CTAs
// or clusters); threads 0 -> the default CTA size of the policy.
int lanczos_threads(int requested, int precision);
int lanczos_smem_bytes(const Plan& P, int nshift, int precision);
cudaError_t lanczos_capacity(const Plan& P, int nshift, int threads, int precision, int* owners);
cudaError_t launch_lanczos(const Plan& P, const LanczosArgs& a, int owners, int precision, int threads,
                           cudaStream_t st);
// Packed launch of several systems sharing the cluster size of P (items, start on the device).
cudaError_t lanczos_batch_capacity(const Plan& P, int threads, int precision, int smem, int* owners);
cudaError_t launch_lanczos_batch(const Plan& P, const BatchItem* items, const int* start, int nitems, int* counter,
                                 int owners, int precision, int threads, int smem, cudaStream_t st);
int solve_smem_bytes(const Plan& P, int nshift);
int apply_smem_bytes(const Plan& P, int es);
cudaError_t solve_grid(const Plan& P, int nshift, int nrhs, int* grid);
cudaError_t launch_solve(const Plan& P, const SolveArgs& a, int grid, cudaStream_t st);
cudaError_t apply_owners(const Plan& P, int precision, int* owners);
// scratch: 2 n_pw complex128 slots per owner
cudaError_t launch_apply(const Plan& P, int nvec, const double2* x, double2* y, const double2* z, int project,
                         double2* scratch, int owners, int precision, cudaStream_t st);
// Im z_rj = eta_s[j] when eta_s is given, else eta; the certificate divides by |Im z|;
// bvec [nrhs][npw] = -P_c rhs when given (else the kernel projects rhs itself).  precision
// selects the arithmetic of the H application inside (FP64, else float-float); clean:
// replace each checked x by P_c x first (x is then written); scratch: 2 n_pw complex128 slots
// per owner.
cudaError_t residual_owners(const Plan& P, int precision, int* owners);
cudaError_t launch_residual(const Plan& P, int nrhs, int nshift, const int* list, int nlist, const double2* rhs,
                            const double* e_ref, const double* omega, double eta, const double2* x, double2* scratch,
                            double* rel, double* cert, double2* store, int owners, cudaStream_t st,
                            const double* eta_s = nullptr, const double2* bvec = nullptr,
                            int precision = SGW_PREC_FP64, int clean = 0);
// b[r] = -P_c rhs[r] (FP64) for r < nrhs; a precomputed bvec lets the residual kernel skip it.
cudaError_t launch_project_rhs(const Plan& P, int nrhs, const double2* rhs, double2* b, cudaStream_t st);
// dn[po][pi][j] += weight sum_v sum_g conj(R[v n_p + po][g]) (X[v n_p + pi][j][g] + X[v n_p + pi][nw + j][g])
// (Eq. 5 in reciprocal space); R [n_v n_p][npw], X [n_v n_p][2 nw][npw], dn [n_p][n_p][nw].
cudaError_t launch_density(int n_v, int n_p, int nw, int npw, const double2* R, const double2* X, double weight,
                           double2* dn, cudaStream_t st);
// epsilon^-1 and W-bar per frequency (Eq. 4, 9) from dn [n][n][nw] and q + G [n][3] (device);
// einv may be null; *bad (device int) is set when a frequency's epsilon is singular.
int screening_smem_bytes(int n);
cudaError_t launch_screening(int n, int nw, const double2* dn, const double* qg, double inv_vol, double r_cut,
                             double2* einv, double2* wbar, int* bad, cudaStream_t st);
// AAA approximation of nfun functions sampled at the m points z (f [nfun][m], m <= 128,
// mmax <= 32), evaluated at ze [ne] into re [nfun][ne]; degree [nfun] (support points) may be
// null; *bad is set when a function has a non-finite sample.
cudaError_t launch_aaa(int nfun, int m, const double2* z, const double2* f, double tol, int mmax, int ne,
                       const double2* ze, double2* re, int* degree, int* bad, cudaStream_t st);
// rhs[c][g] = 1 if g == cols[c] else 0 ([ncol][npw]); the right-hand sides of Eq. 2.
cudaError_t launch_unit_rhs(const int* cols, int ncol, int npw, double2* rhs, cudaStream_t st);
cudaError_t launch_pair_axpy(int nlist, const int* list, int npw, const double2* d, double2* x, cudaStream_t st);
cudaError_t resident_grid(const void* kernel, int smem, int* grid, int threads = kThreads);
cudaError_t launch_to_f32(const double* src, size_t n, float* dst, cudaStream_t st);

}  // namespace sgw
