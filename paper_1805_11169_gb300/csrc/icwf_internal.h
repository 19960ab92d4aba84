// Internal declarations shared by the host orchestration (api.cpp) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/icwf.h"

namespace icwf {

// Status word bits (device int32 at status[0]); counters follow.
enum : int {
  ST_NONFINITE = 1,     // NaN/Inf seen in a velocity, coefficient or matrix
  ST_CHOL = 2,          // Cholesky pivot <= 0
  ST_TIMEOUT = 4,       // bounded wait gave up
  ST_ARG = 8            // kernel saw an out-of-range size
};
// STATUS_WAITLIM: 0 = the compiled-in limits of the spin waits on global flags; k > 0 = those waits
// give up after k - 1 polls (set by icwf_set_wait_limit, a diagnostic for the timeout path).
enum : int { STATUS_FLAGS = 0, STATUS_CLAMPED = 1, STATUS_TICKET = 2, STATUS_WAITLIM = 3,
             STATUS_WORDS = 8 };

// ---------------------------------------------------------------- launch descriptors

// Device view of one ICWF job's state, passed by value to kernels.  Matrices are row-major
// N x N complex128 ([a*N + b], a = bra row, b = ket column).  CWFs are column-major:
// psi[a*nx + i] = psi_a(x_i), chi[a*nR + j] = chi_a(R_j); complex128 (FP64 mode) or complex64.
struct JobView {
  int N, nx, nR, K, logx, logR;
  double x_min, dx, R_min, dR, inv_mx, inv_mR, dt, eps;
  const double* V;        // nx*nR row-major
  const void* Vt;         // the same table in the CWF storage precision (float or double)
  const double* U;        // K*nx  (u_k contiguous)
  const double* W;        // K*nR
  const double* sig;      // K
  const double* v1;       // nx
  const double* v2;       // nR
  void* psi;              // N*nx complex
  void* chi;              // N*nR complex
  double* x;              // N (positions at the current time)
  double* R;
  double* xo;             // N (positions at the previous time; midpoints use both)
  double* Ro;
  double* px;             // K*N: u_k(x_b)
  double* pR;             // K*N: w_k(R_b)
  double* d;              // N: V(x_b, R_b) from the factors
  const void* kinx;       // nx bit-reversed kinetic phases / nx
  const void* kinR;
  const void* twx;        // nx/2 twiddles exp(-2 pi i k / nx)
  const void* twR;
  int* status;
  float* scratch_f32;     // 2N floats (mixed modes: C in FP32 for the velocity kernel), or NULL
};

// Per-kernel-family timing hook (api.cpp implements it).
struct Prof;

// ---------------------------------------------------------------- kernels (launchers)

// a4: velocities (Eq. v1/v2), Euler positions (clamped), pinned factor values at the new
// positions.  T = CWF storage type.
template <typename T> void launch_velocity(const JobView& j, const double2* C, cudaStream_t s);

// a1-a3: Strang split-operator step of every psi_a (pinned at the R midpoint) and chi_a (pinned
// at the x midpoint).  mode 0 = propagate; mode 1 = apply the kinetic operator only (writes to
// out, diagnostic).
// threads: CTA size (a power of two in [64, 512], chosen per shape by the autotuner in api.cpp).
template <typename T> void launch_propagate(const JobView& j, int threads, cudaStream_t s);
template <typename T> void launch_kinetic(const JobView& j, void* out_psi, void* out_chi,
                                          cudaStream_t s);

// Grouped launches over the live jobs of a serving pool (one precision per group).  One entry per
// job: its view, its coefficients, the clamp bounds and inverse masses the velocity step uses, and
// where the job's work items start in the group's item lists (jobs sorted by both).
struct GroupJob {
  JobView j;
  const double2* C;
  double xlo, xhi, Rlo, Rhi;   // first and last cell centres: positions are clamped to them
  float inv_mx_f, inv_mR_f;    // 1/m in FP32 (the mixed modes' velocity arithmetic)
  int traj0;                   // first trajectory item of the job (velocities; prefix sum of N)
  int cwf0;                    // first CWF item of the job (propagation; prefix sum of 2N)
};
// The job's entry with traj0 = cwf0 = 0; bounds and masses as launch_velocity computes them.
GroupJob group_job(const JobView& j, const double2* C);
// Index of the job whose item range holds `item` (0 <= item < the group's total): binary search
// over the jobs' starts (traj0, or cwf0 with `cwf`), which increase strictly since every job has
// N >= 1.  Host and device code.
__host__ __device__ inline int group_find(const GroupJob* __restrict__ g, int njobs, int item,
                                          bool cwf) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int start = cwf ? g[mid].cwf0 : g[mid].traj0;
    if (start <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// Adds two kernel nodes to `graph`: a persistent velocity kernel over every trajectory of the
// njobs jobs in `table` (device memory, njobs >= 1, T = their CWF storage type), then a persistent
// propagation kernel over every CWF of them (a Strang step, as launch_propagate), which depends on
// the first; the first depends on deps[0..ndeps).  Each CTA loops over work items (a warp per
// trajectory, a CTA of `threads` per CWF) with a stride of the grid, which is one wave at full
// occupancy, at most max_ctas CTAs if max_ctas > 0.  nmax = the largest nx or nR of the group.
// *last receives the propagation node.  False if a node cannot be added.
template <typename T>
bool add_group_nodes(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                     const GroupJob* table, int njobs, int total_traj, int total_cwf, int nmax,
                     int threads, int max_ctas, cudaGraphNode_t* last);

// a5 (FP64): S = S1 o S2 and Heff from the rank-K factors at the current positions.
void launch_assemble_fp64(const JobView& j, double2* S, double2* H, cudaStream_t s);

// Generic Gram G = scale * A^H diag(dg) B (A, B column-major n x N complex of type T, dg may be
// NULL for identity); output N x N complex128 row-major.
template <typename T> void launch_gram(const void* A, const void* B, const double* dg, int n,
                                       int N, double scale, double2* G, cudaStream_t s);

// Elementwise H = T1 o S2 + S1 o T2 + sum_k sig_k A_k o B_k + V1 o S2 + S1 o V2 (diagnostic).
void launch_combine_h(int N, const double2* T1, const double2* T2, const double2* S1,
                      const double2* S2, const double2* V1, const double2* V2, const double2* W,
                      double2* H, cudaStream_t s);
void launch_hadamard_acc(int N, double sig, const double2* A, const double2* B, double2* W,
                         cudaStream_t s);

// a6: regularised Cholesky and RK4.
// A[m] = (1-theta_m) S0 + theta_m S1 + eps I for the batch of matrices m (full N x N).
void launch_shift_mix(int N, const double2* S0, const double2* S1, double eps, double theta,
                      double2* A, cudaStream_t s);
// Right-looking blocked Cholesky of nbatch <= 2 matrices in place (lower triangle = L); inv[m]
// receives the N reciprocal pivots 1/L_cc and D[m] (N x 32 complex) the inverses of the 32 x 32
// diagonal blocks.  With emu_scratch (herk_emu_scratch_bytes(N) bytes) the trailing updates run
// on the tensor cores in emulated FP64 (k_herk_emu.cu), else with FP64 FMAs.  Returns the number
// of kernels launched.
int launch_cholesky(int N, double2* const* A, double* const* inv, double2* const* D, int nbatch,
                    int* status, cudaStream_t s, void* emu_scratch = nullptr, size_t emu_bytes = 0);
// Trailing update A_rc -= L_r,jb L_c,jb^H (c <= r, both past block column jb) of nbatch <= 2
// matrices in emulated FP64 on the tensor cores: the panel's digit planes (unless digits_done:
// the panel solve wrote them) and the update.  False if the scratch is too small or a tensor map
// cannot be encoded (nothing launched then).
size_t herk_emu_scratch_bytes(int N);
struct EmuPlanes { void* planes[2]; int* ex[2]; int rpad; };   // digit planes inside the scratch
EmuPlanes herk_emu_planes(int N, void* scratch);
bool launch_herk_emu(int N, int jb, double2* const* A, int nbatch, void* scratch, size_t bytes,
                     bool digits_done, int* status, cudaStream_t s);
void herk_emu_attributes();
// y = ((1-theta) H0 + theta H1) (C + c * kp)      (kp may be NULL)
void launch_matvec(int N, const double2* H0, const double2* H1, double theta, const double2* C,
                   const double2* kp, double c, double2* y, cudaStream_t s);
// L z = y (forward) then L^H w = z (backward); out = scale_i * w with scale_i = -i when
// minus_i, else 1.  work needs 2N complex; flags holds 2*ceil(N/32) block flags followed by the
// 2 tickets (the launcher zeroes all of them first, so any fixed epoch > 0 works and a captured
// sequence can be replayed); `tickets` is unused.
void launch_chol_solve(int N, const double2* L, const double2* D, const double2* y, double2* work,
                       double2* out, bool minus_i, unsigned* flags, unsigned* tickets,
                       unsigned epoch, int* status, cudaStream_t s);
// Mixed modes: the same factorisation and solves in double-float arithmetic (k_linalg_df.cu).
// A, L and D hold complex double-floats (16 bytes each, the size of a complex128), inv holds
// double-float reciprocal pivots (8 bytes each); y and out are complex128.
void launch_shift_mix_df(int N, const double2* S0, const double2* S1, double eps, double theta,
                         void* A, cudaStream_t s);
// One launch per block column with look-ahead; ctl holds chol_ctl_words(N) words of ticket and
// flag state (the launcher zeroes it).
int launch_cholesky_df(int N, void* const* A, void* const* inv, void* const* D, int nbatch,
                       unsigned* ctl, int* status, cudaStream_t s);
size_t chol_ctl_words(int N);
void launch_chol_solve_df(int N, const void* L, const void* D, const double2* y, void* work,
                          double2* out, bool minus_i, unsigned* flags, unsigned* tickets,
                          unsigned epoch, int* status, cudaStream_t s);
// C += dt/6 (k1 + 2 k2 + 2 k3 + k4); flags non-finite values.
void launch_rk4_final(int N, double2* C, const double2* k1, const double2* k2,
                      const double2* k3, const double2* k4, double dt, int* status,
                      cudaStream_t s);
void launch_check_finite(int n, const double2* a, int* status, cudaStream_t s);

// a7: observables.
// Psi[i*nR + j] = sum_a C_a psi_a(x_i) chi_a(R_j)  (complex128 output).
template <typename T> void launch_reconstruct(const JobView& j, const double2* C, double2* Psi,
                                              cudaStream_t s);
// Column / row reductions of Psi: rho_R, rho_x, potential energy, BO projections, FFT kinetic
// energies (partials), then the final deterministic sums into out[0..3] = norm, ekx, ekR, epot.
// part needs 2 nR + nx doubles, proj n_states * nR complex; twx/twR are FP64 twiddles.
void launch_obs_lines(const JobView& j, const double2* Psi, const double* phi, int n_states,
                      double* rho_x, double* rho_R, double2* proj, double* part, double* out,
                      double* pop, double* decoh, const double2* twx, const double2* twR,
                      cudaStream_t s);

// Initial projection b_a = dx dR sum_ij conj(psi_a(x_i) chi_a(R_j)) Psi0[i, j] (FP64 CWFs).
void launch_init_projection(int N, int nx, int nR, double dx, double dR, const double2* psi,
                            const double2* chi, const double2* Psi0, double2* b, cudaStream_t s);
// Convert complex128 -> complex64.
void launch_to_c64(size_t n, const double2* in, float2* out, cudaStream_t s);

// Everything the observables kernels need from a handle (filled by handle_obs_view in api.cpp).
struct ObsView {
  JobView j;
  const double2* C;
  const double* phi;
  int n_states;
  bool mixed;
  bool initialised;
  const double2* twx_d;
  const double2* twR_d;
  cudaStream_t stream;
  int device;
  double t;
};
bool handle_obs_view(icwf_handle h, ObsView* v);
void handle_set_error(icwf_handle h, const char* msg);

// Mixed-precision assembly on the tensor cores (tcgen05); returns false if unsupported sizes.
// exact_s: S from launch_gram_s (exact Grams of fixed-point CWFs), else from the split products.
bool launch_assemble_tc(const JobView& j, int kind, bool exact_s, double2* S, double2* H,
                        void* scratch, size_t scratch_bytes, cudaStream_t s);
size_t assemble_tc_scratch_bytes(int N, int nx, int nR, int K);
// S = S1 o S2 as exact Grams of 4-digit fixed-point complex64 CWFs on the tensor cores
// (k_gram_s.cu); scratch of gram_s_scratch_bytes.  Returns false if it does not fit.
bool launch_gram_s(const JobView& j, double2* S, void* scratch, size_t bytes, cudaStream_t s);
size_t gram_s_scratch_bytes(int N, int nx, int nR);

}  // namespace icwf
