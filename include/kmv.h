/*
 * kmv.h - matrix-free squared-exponential kernel products for determinant-free
 * fully Bayesian Gaussian-process regression, on one GB300 (sm_103a).
 *
 * The operator is A(theta) = K(theta) + sigma^2 I (Eq. kerdef) with the
 * squared-exponential kernel of Sec. 1,
 *     K_ij = alpha * exp(-1/2 * sum_k (x_ik - x_jk)^2 / l_k^2),
 * isotropic (one l) or ARD (one l_k per input dimension).  K is never stored:
 * every call recomputes its entries tile by tile, so device memory stays
 * linear in N.
 *
 * Hyperparameters are FP64 log parameters, one row per (instance, chain):
 *     theta[s, :] = [log alpha, log l_1 .. log l_k, log sigma^2],
 *     n_theta = 2 + (ard ? d : 1),   s = b * chains + c.
 *
 * Kernel family of Sec. 4 (kmv_points.cheb = N_cheb >= 1): the squared
 * exponential with a non-stationary vertical scale,
 *     K_ij = exp(C(x_i)) exp(C(x_j)) exp(-1/2 sum_k (x_ik - x_jk)^2 / l_k^2),
 *     C(x) = sum_t Theta_t T_{t_1}(x_1) .. T_{t_d}(x_d),  t in [0, N_cheb)^d,
 * T_n the Chebyshev polynomials of the first kind (points meant to lie in
 * [-1, 1]^d), with
 *     theta[s, :] = [Theta (N_cheb^d, row-major, t_1 slowest), log l_1 .. log l_k,
 *                    log sigma^2],   n_theta = N_cheb^d + (ard ? d : 1) + 1.
 * Every entry point takes this family; gradients give d/dTheta_t =
 * sum_ij (G V^T)_ij (T_t(x_i) + T_t(x_j)) K_ij in place of d/dlog alpha.
 *
 * Common conventions
 *   - Every pointer documented DEVICE is caller-owned device memory on the
 *     handle's device; HOST pointers are read during the call only.  The
 *     library never frees caller memory.  It owns only its handle workspace,
 *     which grows on demand (cudaMalloc) and is released by kmv_destroy.
 *   - Point sets: instances are concatenated along rows; kmv_points.offsets
 *     (HOST, n_inst + 1 entries, offsets[0] = 0, non-decreasing) delimits
 *     instance b as rows [offsets[b], offsets[b+1]).  Empty instances are
 *     allowed.  N_total = offsets[n_inst].
 *   - Vectors: per-chain arrays are (chains, N_total, m) row-major FP32; the
 *     rows of chain c of instance b are the rows of that instance.
 *   - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t,
 *     NULL = legacy default stream) unless stated otherwise.
 *   - Errors: argument errors return KMV_EINVAL synchronously before any
 *     launch; CUDA errors return KMV_ECUDA; kmv_last_error() gives a message.
 *     Per-system numerical failures (a solve that did not converge, a
 *     non-finite energy) are reported in the caller's chain_status array.
 *     No call traps or aborts.
 *   - A handle is not thread-safe; use one handle per host thread.  Its
 *     workspace is reused by successive calls, so calls on different streams
 *     must be ordered by the caller.
 *   - While `stream` is being captured into a CUDA graph no call allocates:
 *     a call whose workspace (or scratch of the FP32 product, which small
 *     point sets split over more CTAs) is not yet large enough returns
 *     KMV_EINVAL.  Make the same call once before capturing.
 */
#ifndef KMV_H
#define KMV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KMV_OK = 0,
  KMV_EINVAL = 1,       /* bad argument (null pointer, size, layout) */
  KMV_ENOMEM = 2,       /* workspace allocation failed */
  KMV_ECUDA = 3,        /* a CUDA runtime call or launch failed */
  KMV_ENOTCONV = 4,     /* per-system status: solve hit cg_maxiter */
  KMV_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
  KMV_ENONFINITE = 6,   /* per-system status: non-finite value met */
  KMV_EUNSUPPORTED = 7  /* shape or precision not built in this library */
} kmv_status;

typedef enum {
  /* Plain FP32 on the FMA/MUFU pipes: direct differences, FP32 exp2, FP32
   * products folded into FP64 accumulators every 512 columns.  Relative
   * error against FP64 <= 1e-5 on outputs, <= 1e-4 on gradients. */
  KMV_FP32 = 0,
  /* Tensor-core form (tcgen05).  Points are centred per instance (midrange,
   * exact for a stationary kernel).  Products: cross term X_I X_J^T in BF16
   * with a hi/lo split (hi.hi + hi.lo + lo.hi; a three-way split for m <= 2)
   * and the row biases folded into the same contraction, exp2 in FP32
   * registers, P.V in FP16 (FP32 on the FMA pipe for m <= 2) with FP32
   * accumulation over 4096 columns, folded exactly (TwoSum pairs) into FP64
   * partials; relative error against FP64 <= 2e-3.  For m <= 2 and d <= 17
   * the probabilities stay FP32 and the product has FP32 accuracy.
   * Adjoint: the exponent and G.V from F16 hi/lo operands, Q = W o K0 kept
   * exactly as two F16 parts, feature sums accumulated over 256 columns and
   * folded exactly into FP64 partials; gradients to 1e-4 relative like
   * KMV_FP32.  The adjoint needs
   * |x_k - c_k| < 200 l_k and sum_k (x_k - c_k)^2 / l_k^2 < 2^16 / log2(e)
   * (c the centre); beyond, its gradients are NaN (use KMV_FP32). */
  KMV_BF16_HILO = 1
} kmv_precision;

typedef struct kmv_handle_s* kmv_handle;

typedef struct {
  int32_t n_inst;          /* number of independent GP instances, >= 1 */
  const int64_t* offsets;  /* HOST, n_inst + 1 row offsets (see above) */
  int32_t d;               /* input dimension, 1 <= d <= 64 */
  int32_t ard;             /* 0: isotropic kernel, 1: one lengthscale per dimension */
  const float* x;          /* DEVICE, (N_total, d) row-major input points */
  int32_t cheb;            /* 0: the SE kernel of Sec. 1; N_cheb in [1, 32]: the
                              Chebyshev-amplitude family above (N_cheb^d <= 1024,
                              d <= 8 when N_cheb >= 2) */
} kmv_points;

/* Create a handle bound to CUDA device `device` (made current by every call). */
kmv_status kmv_create(kmv_handle* out, int device);
/* Free the handle and its workspace; synchronises the device first. */
kmv_status kmv_destroy(kmv_handle h);
const char* kmv_status_string(kmv_status s);
/* Last error message recorded on this handle ("" if none). */
const char* kmv_last_error(kmv_handle h);
/* Workspace bytes currently held by the handle. */
int64_t kmv_workspace_bytes(kmv_handle h);

/*
 * kmv_forward - Y = A(theta) V (+ col_shift o V), the matrix-free product of
 * Eq. kerdef; col_shift gives the shifted operators A + lambda_p I of Eq. pex.
 *
 *   chains     1..65535 independent hyperparameter sets per instance (the
 *              limit holds for every entry point).
 *   theta      DEVICE FP64 (n_inst * chains, n_theta).
 *   V          DEVICE FP32 (chains, N_total, m), m >= 1.
 *   col_shift  DEVICE FP32 (m) or NULL: column c uses A + col_shift[c] I.
 *   Y          DEVICE FP32 (chains, N_total, m), written (must not alias V).
 *   Y64        DEVICE FP64 (chains, N_total, m) or NULL: the same result before
 *              rounding to FP32 (used for FP64 energy accumulation).
 * Work: sum_b N_b^2 * chains kernel entries ("pairs").
 */
kmv_status kmv_forward(kmv_handle h, const kmv_points* pts, int32_t chains,
                       const double* theta, const float* V, int32_t m,
                       const float* col_shift, float* Y, double* Y64,
                       kmv_precision prec, void* stream);

/*
 * kmv_backward - adjoint of L_s = sum_{i in b, k} G[c,i,k] (A(theta_s) V)[c,i,k]
 * for each system s = (b, c); the quadratic-form gradient of primitive (3),
 * Sec. 3.2.1, generalised to many vectors.
 *
 *   grad_theta DEVICE FP64 (n_inst * chains, n_theta), overwritten with dL_s/dtheta_s:
 *                d/dlog alpha   = sum_ij (G V^T)_ij K_ij
 *                d/dlog l_k     = sum_ij (G V^T)_ij K_ij (x_ik - x_jk)^2 / l_k^2
 *                                 (isotropic: summed over k)
 *                d/dlog sigma^2 = sigma^2 sum_i G_i . V_i
 *   grad_V     DEVICE FP32 (chains, N_total, m) or NULL: dL/dV = A G.
 * K entries are recomputed, never stored.  The FP64 reduction over tiles is
 * in a fixed order, so results are bitwise reproducible.
 */
kmv_status kmv_backward(kmv_handle h, const kmv_points* pts, int32_t chains,
                        const double* theta, const float* V, const float* G,
                        int32_t m, double* grad_theta, float* grad_V,
                        kmv_precision prec, void* stream);

/*
 * kmv_cg_solve - solve A(theta_s) x = rhs for every system s by conjugate
 * gradients (primitive (1) of Sec. 3.2.1; Eq. xtheta), stopping a system when
 * ||r|| <= tol ||rhs|| (Sec. 4 uses tol = 1e-6).
 *
 *   rhs          DEVICE FP32 (N_total) shared by all chains if rhs_per_chain == 0,
 *                else (chains, N_total).
 *   x            DEVICE FP32 (chains, N_total): initial guess if warm_start != 0,
 *                otherwise ignored; overwritten with the solution.
 *   chain_status DEVICE int32 (n_inst * chains): KMV_OK or KMV_ENOTCONV.
 *   iters        DEVICE int32 (n_inst * chains) or NULL: iterations used.
 * KMV_BF16_HILO with d <= 17 runs CG directly on the tensor-core one-column
 * product, whose probabilities are FP32 (FP32-accurate like KMV_FP32).  For
 * d > 17 it solves by mixed-precision iterative refinement: the residual
 * rhs - A x is formed with the FP32 operator and each correction is solved by
 * CG with the tensor-core operator (to 1e-3), so the result meets `tol`
 * against the FP32 operator or reports KMV_ENOTCONV; `iters` then counts the
 * tensor-core CG iterations.  With a Nystrom preconditioner set on the handle
 * (kmv_set_preconditioner) the CG, and the refinement's inner CG, are
 * preconditioned.
 * Outside stream capture, the call synchronises `stream` every few iterations
 * to test convergence on the host.  While `stream` is being captured into a
 * CUDA graph, the iterations after the first are recorded as a conditional
 * WHILE node whose condition a device kernel sets from the count of systems
 * still active, so a replay stops at convergence (or at cg_maxiter) exactly
 * like the eager solve, with no host synchronisation (the refined d > 17
 * solve records three refinement steps).  Under capture
 * nothing may be allocated: make the same call (same shapes, same stream
 * device) once before capturing, and leapfrog_step / kmv_energy likewise.
 */
kmv_status kmv_cg_solve(kmv_handle h, const kmv_points* pts, int32_t chains,
                        const double* theta, const float* rhs, int32_t rhs_per_chain,
                        float* x, double tol, int32_t maxiter, int32_t warm_start,
                        int32_t* chain_status, int32_t* iters,
                        kmv_precision prec, void* stream);

/*
 * leapfrog_step - one drift-kick-drift step of Sec. 3.2.2 for every chain:
 *     theta_h = theta + dt/2 pi
 *     x       = A(theta_h)^{-1} y                         (kmv_cg_solve, cold start)
 *     F       = grad S(theta_h) + d/dtheta [ -x^T A x / 2 + phi^T A phi / 2 ]
 *               (the frozen-x force of Eq. u, via kmv_backward with
 *                V = [x, phi], G = [-x/2, phi/2])
 *     pi     <- pi - dt F
 *     theta  <- theta_h + dt/2 pi
 * Components with free_mask[p] == 0 receive neither drift nor kick.
 *
 *   y            DEVICE FP32 (N_total) observations.
 *   phi          DEVICE FP32 (chains, N_total) auxiliary Gaussian variables.
 *   theta, pi    DEVICE FP64 (n_inst * chains, n_theta), updated in place.
 *   prior_mu, prior_prec DEVICE FP64 (n_theta) or both NULL (flat prior,
 *                S = 0); otherwise S = sum prec (theta - mu)^2 / 2.
 *   free_mask    DEVICE uint8 (n_theta) or NULL (all free).
 *   x_work       DEVICE FP32 (chains, N_total): receives x.
 *   chain_status DEVICE int32 (n_inst * chains): KMV_OK, or KMV_ENOTCONV when
 *                the solve failed (theta/pi then hold theta_h / the un-kicked pi;
 *                the caller must reject the trajectory).
 *   cg_iters     DEVICE int32 (n_inst * chains) or NULL.
 * prec selects the operator of the solve (see kmv_cg_solve) and the adjoint of
 * the force.  The force's two quadratic forms are sums of N^2 terms that can
 * cancel to a small fraction of their size (x = A^-1 y oscillates); the
 * KMV_BF16_HILO adjoint keeps every pair's term near FP32 accuracy, so its
 * force agrees with the FP32 one there too.
 */
kmv_status leapfrog_step(kmv_handle h, const kmv_points* pts, int32_t chains,
                         const float* y, const float* phi, double* theta, double* pi,
                         double dt, const double* prior_mu, const double* prior_prec,
                         const uint8_t* free_mask, double cg_tol, int32_t cg_maxiter,
                         float* x_work, int32_t* chain_status, int32_t* cg_iters,
                         kmv_precision prec, void* stream);

/*
 * kmv_implicit_step - one implicit midpoint step of Sec. 3.2.3 for every chain:
 * the (theta_1, pi_1, x) of Eq. implicitsystem,
 *     theta_1 = theta_0 + dt (pi_0 + pi_1)/2,
 *     pi_1    = pi_0 - dt F(theta_bar, x),   theta_bar = (theta_0 + theta_1)/2,
 *     A(theta_bar) x = y,
 * with F the frozen-x force of leapfrog_step, found as the fixed point of the
 * map Phi of Eq. Phi by Anderson acceleration with depth aa_depth (App. B; the
 * paper uses 10), theta, pi and x taken as one vector.  Phi's linear part uses
 * R = P^{-1} / c when a Nystrom preconditioner is set (kmv_set_preconditioner),
 * else R = I / c, c = 1.05 x a 20-step power estimate of rho(P^{-1} A(theta_0))
 * (resp. rho(A(theta_0))), so that the plain iteration contracts.  A system
 * stops when every theta, pi component of z - Phi(z) is <= tol (1 + max
 * |Phi(z)|) and |y - A(theta_bar) x| <= tol |y|, or that residual is below
 * 1e-3 |y| and has not halved in 8 aa_depth iterations (the floor of the FP32
 * product, about 2^-24 |A| |x|, can lie above tol |y| on ill-conditioned systems);
 * theta, pi and x_work then hold Phi(z) of that iteration.
 *
 *   theta, pi    DEVICE FP64 (n_inst * chains, n_theta): in theta_0, pi_0; out
 *                theta_1, pi_1.
 *   x_work       DEVICE FP32 (chains, N_total): in the starting x (e.g. the last
 *                step's), out x at the midpoint.
 *   aa_depth     1..16; maxiter >= 1 iterations (each one product, one FP32 adjoint).
 *   chain_status DEVICE int32: KMV_OK, KMV_ENOTCONV (maxiter reached: theta,
 *                pi hold the last iterate; reject), KMV_ENONFINITE.
 *   iters        DEVICE int32 (n_inst * chains): iterations taken.
 *   prior_mu, prior_prec, free_mask as in leapfrog_step.  Both forms (prec)
 *   take FP32 products and the FP32 adjoint here: the iteration measures the
 *   true residual y - A x, which the tensor-core product's rounding keeps
 *   above tol on ill-conditioned systems.
 * The Metropolis test needs A(theta_1)^{-1} y afterwards (kmv_energy).
 */
kmv_status kmv_implicit_step(kmv_handle h, const kmv_points* pts, int32_t chains,
                             const float* y, const float* phi, double* theta, double* pi,
                             double dt, const double* prior_mu, const double* prior_prec,
                             const uint8_t* free_mask, int32_t aa_depth, double tol,
                             int32_t maxiter, float* x_work, int32_t* chain_status,
                             int32_t* iters, kmv_precision prec, void* stream);

/*
 * kmv_energy - the Hamiltonian of Sec. 3.2 per chain, accumulated in FP64:
 *     U = S(theta) + y^T x / 2 + phi^T A phi / 2,  x = A(theta)^{-1} y   (Eq. U)
 *     H = U + pi^T pi / 2                                            (M = I)
 *   pi       DEVICE FP64 (n_inst * chains, n_theta) or NULL (H = U).
 *   H        DEVICE FP64 (n_inst * chains), written.
 *   terms    DEVICE FP64 (n_inst * chains, 3) or NULL: [S, y^T x / 2, phi^T A phi / 2].
 *   Other arguments as in leapfrog_step.  prec selects the operator used by
 *   the solve and the product; KMV_FP32 is the accurate form meant for the
 *   Metropolis test.
 */
kmv_status kmv_energy(kmv_handle h, const kmv_points* pts, int32_t chains,
                      const float* y, const float* phi, const double* theta,
                      const double* pi, const double* prior_mu, const double* prior_prec,
                      double cg_tol, int32_t cg_maxiter, float* x_work,
                      double* H, double* terms, int32_t* chain_status, int32_t* cg_iters,
                      kmv_precision prec, void* stream);

/*
 * kmv_accept - the Metropolis test of Algorithm 1 for every system: accept iff
 * status[s] == KMV_OK (status may be NULL), both energies are finite and
 * log u[s] <= H_old[s] - H_new[s] (the event u <= min(1, exp(H_old - H_new))
 * for u in (0, 1]); a rejected system's theta gets theta_old back.
 *   H_old, H_new, u  DEVICE FP64 (n_sys); u the caller's U(0, 1] draws.
 *   theta_old        DEVICE FP64 (n_sys, n_theta); theta DEVICE FP64, in/out.
 *   accepted         DEVICE int32 (n_sys): 1 accepted, 0 rejected.
 * kmv_status_merge - dst[s] = src[s] where dst[s] is KMV_OK and src[s] is not
 * (collects the first failure of a trajectory's steps for kmv_accept).
 * Neither needs a handle; both are stream-ordered on `stream`.
 */
kmv_status kmv_accept(int32_t n_sys, int32_t n_theta, const double* H_old, const double* H_new,
                      const double* u, const int32_t* status, const double* theta_old,
                      double* theta, int32_t* accepted, void* stream);
kmv_status kmv_status_merge(int32_t n, const int32_t* src, int32_t* dst, void* stream);

/*
 * kmv_phi_refresh - the Gibbs draw of the auxiliary variable of Sec. 3.1,
 * phi = A(theta_s)^{-1/2} xi for every system s, by the pole expansion of
 * App. A (Eq. pex):  phi = sum_p w_p (A + lambda_p I)^{-1} xi, p = 1..n_poles,
 * with weights and shifts from Jacobi elliptic functions on the spectral
 * interval [sigma_s^2, M_s], M_s = 1.01 max_i (A 1)_i (the largest row sum
 * bounds lambda_max because K0 >= 0 entrywise; 1% covers rounding).  The
 * n_poles shifted systems of every system share xi, so one CG sequence on the
 * smallest shift carries them all (multi-shift CG: the shifted iterates follow
 * from its scalars), each shift stopping at cg_tol.  For d > 17 (where its
 * one-column product is not FP32-accurate) the BF16 form then checks every
 * shifted solution with the FP32 operator and polishes those above cg_tol by
 * refinement (FP32 residuals, corrections by a multi-column CG whose one
 * product per iteration applies all the shifts as column shifts).
 *
 *   xi          DEVICE FP32 (chains, N_total): the caller's N(0, I) draw.
 *   phi         DEVICE FP32 (chains, N_total), written (must not alias xi).
 *   n_poles     1..32 (Sec. 3.1 uses 15).
 *   chain_status DEVICE int32 (n_inst * chains): KMV_OK, or the first failure
 *               (KMV_ENOTCONV, KMV_ENONFINITE) among the system's shifted solves.
 *   cg_iters    DEVICE int32 (n_inst * chains) or NULL: the largest iteration count.
 *   poles_out   DEVICE FP64 (n_inst * chains, 2 + 2 n_poles) or NULL:
 *               [sigma^2, M, w_1..w_Np, lambda_1..lambda_Np] per system.
 * Work: one N^2 pass for A 1, then one single-column N^2 product per CG
 * iteration (a system drops out when all its shifts have stopped); the d > 17
 * BF16 check costs one n_poles-column FP32 product per refinement step.
 * cg_iters counts the multi-shift iterations plus the polishing ones.  Allocates workspace; not for use while the
 * stream is being captured (the work plan changes between the two phases).
 */
kmv_status kmv_phi_refresh(kmv_handle h, const kmv_points* pts, int32_t chains,
                           const double* theta, const float* xi, float* phi,
                           int32_t n_poles, double cg_tol, int32_t cg_maxiter,
                           int32_t* chain_status, int32_t* cg_iters, double* poles_out,
                           kmv_precision prec, void* stream);

/*
 * Randomized Nystrom preconditioner (Frangella, Tropp and Udell), which the
 * paper uses for its linear solves (Sec. 3.1, end; Sec. 3.2.3; Sec. 4): a
 * rank-r factorisation K(theta) ~ U diag(lambda) U^T per system, used through
 * the Woodbury form for A = K + sigma^2 I,
 *     P^{-1} = (lambda_r + sigma^2) U (diag(lambda) + sigma^2)^{-1} U^T + (I - U U^T),
 * with sigma^2 taken from the theta of each solve, so one factorisation can
 * serve the solves at later theta (the paper rebuilds it every few updates).
 *
 * kmv_nystrom_build - Y = K Omega (one r-column product without the noise
 * term), nu = sqrt(N_b) 2^-23 |Y|_F, Y_nu = Y + nu Omega, Omega^T Y_nu = L L^T,
 * B = Y_nu L^{-T} = U S W^T, lambda = max(S^2 - nu, 0).
 *   rank        1..128 (the paper uses 5 and 500).
 *   omega       DEVICE FP32 (chains, N_total, rank): the caller's N(0, 1) draws.
 *   U           DEVICE FP32 (chains, rank, N_total), written: the orthonormal
 *               columns, stored column after column.
 *   lam         DEVICE FP64 (n_inst * chains, rank), written, descending.
 *   chain_status DEVICE int32 (n_inst * chains): KMV_OK, or KMV_ENOTCONV when the
 *               r x r Cholesky failed (e.g. an instance with fewer than rank
 *               points); that system then gets lam = 0, U = 0 (P = I).
 * Work: one rank-column N^2 product, O(N rank^2) Gram and U passes, O(rank^3)
 * per system in FP64.  Allocates workspace; not for use during capture.
 *
 * kmv_set_preconditioner - from the next call on, every CG solve on this
 * handle (kmv_cg_solve, leapfrog_step, kmv_energy, both precisions) runs
 * preconditioned CG with pc, until it is called with NULL.  The arrays are the
 * caller's and must stay valid while set; a solve whose layout (n_inst,
 * chains, N_total) differs from pc's returns KMV_EINVAL.  kmv_phi_refresh then
 * solves its shifted systems as preconditioned columns of one multi-column CG
 * (mu = sigma^2 + lambda_p per column: the same factors serve every shift)
 * instead of multi-shift CG, whose shift invariance a preconditioner breaks;
 * that solve takes FP32 products in both forms (the many-column tensor-core
 * product is too coarse to refine the small shifts when sigma^2 << |K|).
 */
typedef struct {
  int32_t rank;
  int32_t n_inst;
  int32_t chains;
  int64_t n_total;
  const float* U;      /* DEVICE (chains, rank, N_total) */
  const double* lam;   /* DEVICE (n_inst * chains, rank) */
} kmv_nystrom;

kmv_status kmv_nystrom_build(kmv_handle h, const kmv_points* pts, int32_t chains,
                             const double* theta, int32_t rank, const float* omega,
                             float* U, double* lam, int32_t* chain_status,
                             kmv_precision prec, void* stream);
kmv_status kmv_set_preconditioner(kmv_handle h, const kmv_nystrom* pc);

/*
 * Kernel timing.  Instrumentation for measuring the library on a device; the
 * paper has no counterpart.  While enabled, every launch of a main product
 * kernel is bracketed by two CUDA events recorded on the call's stream:
 *   KMV_KERNEL_FORWARD  the forward kernel (either precision, including the
 *                       forward pass that kmv_backward runs for grad_V),
 *   KMV_KERNEL_ADJOINT  the adjoint kernel of kmv_backward.
 * The preparation and epilogue kernels around them are not included.  No
 * events are recorded while the stream is being captured into a CUDA graph.
 * kmv_profile_enable(h, on) switches timing on (on != 0) or off and drops
 * the records so far.  kmv_profile_read(h, kind, &total_ms, &launches) waits
 * for the recorded events, returns the summed device time in milliseconds and
 * the number of launches of that kind since the last read or enable, and
 * clears them.  Errors: KMV_EINVAL (null handle or output, unknown kind),
 * KMV_ECUDA (an event could not be read; the others are still summed).
 */
typedef enum { KMV_KERNEL_FORWARD = 0, KMV_KERNEL_ADJOINT = 1 } kmv_kernel_kind;
kmv_status kmv_profile_enable(kmv_handle h, int32_t on);
kmv_status kmv_profile_read(kmv_handle h, int32_t kind, double* total_ms, int64_t* launches);

/*
 * Tile choices of the tensor-core kernels (KMV_BF16_HILO) and an autotuner
 * that picks them per call shape.  The paper has no counterpart (it leaves the
 * GPU kernels to a library); these calls change speed only, never results
 * beyond rounding.
 *
 *   kernel (kmv_tile_kernel):
 *     KMV_TILES_FORWARD      products with m > 2 columns (P.V on the tensor cores)
 *     KMV_TILES_FORWARD_FMA  products with m <= 2 (the CG iterations; P.v on the
 *                            FMA pipe)
 *     KMV_TILES_ADJOINT      the adjoint kernel of kmv_backward
 *   kmv_tiles:
 *     stages        operand-ring stages in shared memory, 2..8 (the adjoint uses
 *                   at most 6); 0 = as many as shared memory holds
 *     items_per_sm  work items per SM the work plan aims at, 1..64 (default 6)
 *     exp_split     0: every exp2 on the MUFU (ex2.approx); 4 or 8: one element
 *                   in 4 (8) by a range-reduced minimax polynomial on the FMA
 *                   pipe (relative error 7.5e-5 for the F16 probabilities of
 *                   KMV_TILES_FORWARD, 1.6e-7 for KMV_TILES_FORWARD_FMA); other
 *                   values round to 0, 4 or 8.  Ignored by the adjoint.
 *
 * kmv_set_tiles sets the default of a kernel kind, used by every shape the
 * autotuner has not recorded; kmv_get_tiles reads it.  Both are host-only and
 * synchronous.  Errors: KMV_EINVAL (null argument, unknown kernel, a value
 * out of range).
 *
 * kmv_autotune times candidate tiles for the shape of (pts, chains, m): the
 * product kernel of kmv_forward with m columns and the adjoint kernel of
 * kmv_backward with m columns, each with every candidate (3 exp splits x 2
 * stage limits x 3 plan densities for the products, 2 x 3 for the adjoint),
 * by CUDA events around the main kernel, and records the fastest for that
 * shape: (kernel, d, m, floor(log2 of the largest instance's size)).  Later
 * calls of that shape run with it; other shapes keep the defaults.  Timing
 * runs on at most the first 65,536 rows of the largest instance with one
 * chain and theta of its first system; values of V and G are synthetic.
 *   cache_path  HOST string or NULL: a text file of recorded shapes, read first
 *               (shapes it holds are not timed again) and rewritten with every
 *               recorded shape afterwards.
 * The call is synchronous, allocates scratch device memory (freed before it
 * returns) and must not be made while `stream` is being captured.  Errors:
 * KMV_EINVAL, KMV_ENOMEM, KMV_ECUDA, KMV_EUNSUPPORTED (no tensor-core form
 * for this shape; nothing recorded).
 */
typedef enum { KMV_TILES_FORWARD = 0, KMV_TILES_FORWARD_FMA = 1, KMV_TILES_ADJOINT = 2 } kmv_tile_kernel;
typedef struct {
  int32_t stages;
  int32_t items_per_sm;
  int32_t exp_split;
} kmv_tiles;
kmv_status kmv_set_tiles(kmv_handle h, int32_t kernel, const kmv_tiles* t);
kmv_status kmv_get_tiles(kmv_handle h, int32_t kernel, kmv_tiles* t);
kmv_status kmv_autotune(kmv_handle h, const kmv_points* pts, int32_t chains, const double* theta, int32_t m,
                        const char* cache_path, void* stream);

/*
 * kmv_backward_noalloc - kmv_backward with KMV_FP32 arithmetic that allocates
 * no device memory and needs no handle.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code
 * whose device memory all belongs to its own pool or arena (memory taken
 * behind the pool's back can make it fail), or loops that cannot take the
 * device-wide synchronisation an allocation may imply.
 *
 *   Arguments and results as in kmv_backward (grad_V may be NULL).
 *   Scratch: a fixed 4 MiB device array inside the library, held by every
 *     device that loads the library until the process exits.  It stores the
 *     row-tile tables and the per-tile FP64 partial sums, so a call must fit
 *       256-byte-aligned (8 (n_inst + 1) + 4 (n_inst + 1) + 12 n_tiles)
 *       + 8 n_tiles * chains * ceil(m / 32) * n_theta  <=  4 MiB,
 *     n_tiles = sum_b ceil(N_b / 128); a call that does not fit returns
 *     KMV_EINVAL before doing any work.  Everything the call reads from the
 *     array it has written first in the same call, so no clearing is needed.
 *   Set-up: the first call on a device, with that device current, looks up
 *     the array's device address (cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   Concurrency: every call on a device shares the one array; calls whose
 *     work overlaps on the GPU (other streams, other host threads) race and
 *     must be ordered by the caller.
 *   Offsets: each call copies pts->offsets (HOST) to the array; the copy is
 *     staged before the call returns, so the host array may change afterwards.
 *   Errors: KMV_EINVAL (bad argument, by the rules of every other entry point,
 *     or scratch limit exceeded), KMV_ECUDA, KMV_EUNSUPPORTED for the
 *     Chebyshev-amplitude family (pts->cheb != 0).
 */
kmv_status kmv_backward_noalloc(const kmv_points* pts, int32_t chains, const double* theta,
                                const float* V, const float* G, int32_t m, double* grad_theta,
                                float* grad_V, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KMV_H */
