/*
 * icwf_exact2d.h -- exact propagation of the full two-coordinate wavefunction on one GB300.
 *
 * The paper judges every ICWF run against the exact solution of its time-dependent Schroedinger
 * equation (Eq. TDSE without vector potential) on the same (x, R) grid: the "exact" curves of
 * the reduced densities, BO populations and decoherence indicators in Figs. 1 and 2.  This
 * solver produces that reference on the GPU with the same potential table, masses, grids and dt
 * as an icwf_params set, by the second-order Strang split
 *   Psi <- e^{-i V dt/2} F^-1 e^{-i (kx^2/2m_x + kR^2/2m_R) dt} F e^{-i V dt/2} Psi,
 * F the 2D discrete Fourier transform on the periodic cell-centred grid.  FP64 throughout.
 *
 * Conventions are those of icwf.h (host pointers, copies, statuses, one stream per handle).
 * Psi is nx * nR complex128, row-major with x the slow index: psi[2*(i*nR + j)] = Re Psi(x_i, R_j).
 */
#ifndef ICWF_EXACT2D_H
#define ICWF_EXACT2D_H

#include "icwf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct icwf_exact2d_ctx* icwf_exact2d;

/* Create from the grid, masses and dt of p (other fields ignored; nx, nR powers of two in
 * [8, 4096]) and V[nx*nR] (row-major V(x_i, R_j), copied).  ICWF_ERR_ARG on bad sizes,
 * ICWF_ERR_OOM if device memory runs out. */
icwf_status icwf_exact2d_create(const icwf_params* p, const double* V, icwf_exact2d* out);

/* Set Psi (nx*nR complex128, copied) and t = 0. */
icwf_status icwf_exact2d_set_state(icwf_exact2d h, const double* psi);

/* BO projectors for the populations (same layout as icwf_set_projectors: phi[n][j][i]
 * = phi_n(x_i; R_j), n < n_states <= 8, real, copied). */
icwf_status icwf_exact2d_set_projectors(icwf_exact2d h, int32_t n_states, const double* phi);

/* Advance n_steps >= 0 Strang steps (ICWF_ERR_STATE before set_state). */
icwf_status icwf_exact2d_step(icwf_exact2d h, int32_t n_steps);

/* Copy Psi out (nx*nR complex128). */
icwf_status icwf_exact2d_get_state(icwf_exact2d h, double* psi);

/* Observables of Psi with the definitions of icwf_obs (rho_x, rho_R, norm, energy with the
 * kinetic terms in Fourier space, pop and decoh if projectors are set; n_clamped = 0). */
icwf_status icwf_exact2d_observables(icwf_exact2d h, icwf_obs* out);

/* Release the handle; NULL is a no-op. */
icwf_status icwf_exact2d_destroy(icwf_exact2d h);

/* One-line description of the last failure on h (or of the last failed create for NULL). */
const char* icwf_exact2d_last_error(icwf_exact2d h);

#ifdef __cplusplus
}
#endif
#endif
