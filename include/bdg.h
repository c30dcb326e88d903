/*
 * libbdg -- dense eigensolver for the static Bogoliubov-de Gennes (BdG)
 * quasiparticle Hamiltonian on one NVIDIA B300 (sm_103a).
 *
 * The problem (arXiv:2310.03341, Eq. (stHpsi), section "Theoretical
 * Framework: TDDFT for Fermions"): find all eigenpairs of
 *
 *         [ h        Delta ] [u_n]       [u_n]
 *         [ Delta^*  -h^*  ] [v_n] = E_n [v_n],      h = T + U(r) - mu,
 *
 * on a periodic Nx x Ny x Nz grid with spacing dx = 1 and hbar = m = 1
 * (section "Numerical setup and implementation").  T is the spectral kinetic
 * operator F^-1 (k^2/2) F with k = 2 pi n / N, n = -N/2 .. N/2-1.  The matrix
 * has dimension N = 2*Nx*Ny*Nz; u_n and v_n are its two halves.
 *
 * Conventions shared by every entry point
 *   - site index s = (ix*Ny + iy)*Nz + iz (z fastest); rows 0..V-1 are u,
 *     rows V..2V-1 are v (V = Nx*Ny*Nz);
 *   - matrices are COLUMN-MAJOR, element (i, j) at a[i + j*ld], complex
 *     numbers interleaved (double2: .x real, .y imaginary);
 *   - all array arguments are caller-owned DEVICE pointers unless marked
 *     "host"; the library never frees them;
 *   - every call is asynchronous on `stream` unless it returns a host scalar
 *     (such calls synchronise `stream` before returning);
 *   - every call returns a status (BDG_OK = 0 or a negative BDG_E* code); it
 *     never aborts or exits.  bdg_last_error() gives the message;
 *   - eigenvalues are returned in ascending order as FP64; eigenvectors are
 *     unit-norm columns with an arbitrary phase (for degenerate eigenvalues
 *     any orthonormal basis of the eigenspace).
 *
 * Precision modes for the reduction and back-transformation (the tridiagonal
 * eigenvalue solve is FP64 in every mode):
 *   BDG_PREC_FP64    all arithmetic in FP64;
 *   BDG_PREC_FP32    reduction/back-transformation in FP32 (complex64);
 *   BDG_PREC_BF16X3  FP32 data with products on the BF16 tensor cores using
 *                    operands split into two bf16 slices (hi + lo, ~16
 *                    significant bits; the three leading slice products),
 *                    FP32 accumulation;
 *   BDG_PREC_BF16X6  the same with three bf16 slices (the full FP32
 *                    significand; the six leading slice products);
 *   BDG_PREC_BF16X9  FP32 data; the large products of stage 1 and of its
 *                    back-transformation run as FP32-accurate products on
 *                    the tensor cores by exact slicing: three 8-bit integer
 *                    slices per operand with a power-of-two scale per
 *                    (column, 64-chunk), the six leading slice pairs,
 *                    integer sums exact within each 64-chunk; the tensor-core
 *                    FP32 accumulation of the two modes above truncates,
 *                    which shows as a ~1e-5 relative bias in long
 *                    accumulations, and this mode never lets it round.
 * Every mode other than BDG_PREC_FP64 is meant to be followed by bdg_refine,
 * which recovers FP64 accuracy; its default cluster threshold follows the
 * mode of the context's last bdg_heev (see bdg_refine).
 */
#ifndef BDG_H
#define BDG_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdg_ctx bdg_ctx;

/* Grid of the periodic box; nx, ny, nz even and >= 2, dx must be 1. */
typedef struct {
    int nx, ny, nz;
    double dx;
} bdg_grid;

enum {
    BDG_OK = 0,
    BDG_EINVAL = -1,        /* invalid argument (sizes, null pointer, odd grid) */
    BDG_ENOMEM = -2,        /* device workspace could not be allocated          */
    BDG_ECUDA = -3,         /* a CUDA runtime call failed                       */
    BDG_ENOCONV = -4,       /* refinement or an iteration did not converge      */
    BDG_ETIMEOUT = -5,      /* a bounded device-side wait gave up               */
    BDG_EUNSUPPORTED = -6   /* size or mode outside what the library supports   */
};

enum { BDG_PREC_FP64 = 0, BDG_PREC_FP32 = 1, BDG_PREC_BF16X3 = 2, BDG_PREC_BF16X6 = 3, BDG_PREC_BF16X9 = 4 };

/* Flag OR-ed into the precision of bdg_heev: the caller asserts that A is a
 * BdG matrix in the layout of bdg_build (n = 2V, u rows then v rows), so
 * that P A P^-1 = -A with P x = C conj(x), C = [[0, I], [-I, 0]]: the
 * partner of an eigenpair (E; u, v) is (-E; conj v, -conj u) (particle-hole
 * symmetry of Eq. (stHpsi)).  When no eigenvalue of the tridiagonal lies
 * within the cluster tolerance of zero, only the upper half of the spectrum
 * and its vectors are computed (bisection, inverse iteration and both
 * back-transformations on n/2 columns) and the lower half is filled with the
 * partners; otherwise the full solve runs. */
#define BDG_HEEV_PH 0x100

/* Create a context bound to CUDA device `device`.  The context owns the
 * device workspace (grown on demand and reused across calls).  One context
 * per host thread.  Returns BDG_OK and *out, or an error (then *out = NULL). */
int bdg_create(int device, bdg_ctx **out);

/* Release the context and its workspace (synchronises the device). */
void bdg_destroy(bdg_ctx *ctx);

/* Text of the last error recorded on this context ("" if none).  The
 * pointer stays valid until the next call on the context. */
const char *bdg_last_error(bdg_ctx *ctx);

/* Build the dense BdG matrix of Eq. (stHpsi):
 *   H = [[h, diag(Delta)], [diag(Delta^*), -h^*]],  h = T + diag(U) - mu,
 * with T the Kronecker sum of the three 1-D spectral kinetic matrices
 * (section "Numerical setup and implementation", kinetic-term equation).
 *   grid   host pointer to the grid description;
 *   U      device, V doubles (real local potential);
 *   Delta  device, V double2 (complex pairing field);
 *   H      device, N x N double2, column-major with leading dimension
 *          ldh >= N; fully overwritten (both triangles).
 * Errors: BDG_EINVAL for a bad grid, null pointers or ldh < N. */
int bdg_build(bdg_ctx *ctx, const bdg_grid *grid, double mu, const double *U,
              const double2 *Delta, double2 *H, int64_t ldh, cudaStream_t stream);

/* Device workspace (bytes) that bdg_heev needs for order n in mode prec. */
int bdg_heev_workspace(bdg_ctx *ctx, int64_t n, int prec, size_t *bytes);

/* All eigenpairs of the Hermitian matrix A (n x n, column-major, lda >= n;
 * both triangles must hold the matrix).  Two-stage reduction (dense -> band
 * -> tridiagonal), FP64 tridiagonal solve (bisection + inverse iteration),
 * two-stage back-transformation -- the 2-stage sequence the paper describes
 * for its eigensolver (section "Performance of the Matrix Diagonalization
 * Algorithm").
 *   A  device, destroyed (used as scratch);
 *   w  device, n doubles, eigenvalues ascending;
 *   Z  device, n x n double2, column-major, ldz >= n; column j is the
 *      eigenvector of w[j].
 * In the reduced-precision modes Z and w carry FP32-level accuracy; call
 * bdg_refine to reach FP64 accuracy.
 * Errors: BDG_EINVAL, BDG_ENOMEM, BDG_ETIMEOUT (a bounded device wait gave
 * up), BDG_EUNSUPPORTED (n beyond the supported size for this mode). */
int bdg_heev(bdg_ctx *ctx, int64_t n, double2 *A, int64_t lda, double *w,
             double2 *Z, int64_t ldz, int prec, cudaStream_t stream);

/* Ogita-Aishima iterative refinement of all eigenpairs of the BdG matrix
 * defined by (grid, mu, U, Delta) -- the matrix is never formed; H*X is
 * applied through its Kronecker-sum structure in FP64.  Each iteration:
 *   R = I - X^H X,  S = X^H H X  (products accurate to FP64 level),
 *   lambda_i = Re S_ii / (1 - Re R_ii),
 *   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)  if
 *          |lambda_i - lambda_j| > omega, else R_ij / 2,
 *   X <- X + X E.
 * omega = 1e-8 * max|lambda|.  Stops when the largest column residual
 * ||H x_i - lambda_i x_i|| / max|lambda| <= tol or after max_iter iterations.
 *   n        must equal 2*nx*ny*nz;
 *   w        device, in: eigenvalue estimates, out: refined (ascending order
 *            is kept; pairs whose estimates cross are reordered with their
 *            vectors);
 *   Z        device n x n double2, in/out;
 *   resid_out, orth_out, iters_out: HOST pointers (may be NULL) receiving the
 *            final max relative residual, max |X^H X - I| and the number of
 *            iterations done.  The stopping test uses the residual alone;
 *            the Gram matrix of the final vectors (one FP64-accurate product)
 *            is formed only when orth_out is not NULL.  Synchronises `stream`.
 * Particle-hole reduction: when the estimates split at zero (w[n/2-1] < 0 <
 * w[n/2], with a gap above 2e-8 max|w|), only the columns n/2..n-1 are
 * refined, using the half-size products X+^H X+, X+^H H X+, X+^T C X+ and
 * X+^T C H X+ (C as for BDG_HEEV_PH).  Columns 0..n/2-1 of Z and w[0..n/2-1]
 * are regenerated as the partners of the upper half on entry and again after
 * every update, so they need not hold the partners on entry.
 * Otherwise all n columns are refined.  bdg_last_modes reports which ran.
 * Method choices (not in the paper): the FP64-accurate products use 4 bf16
 * slices per operand in the first iteration and afterwards 5 (tol >= 5e-11)
 * or 6 (FP64 level, smaller tol); coupled
 * neighbours with |E_ij| above a threshold tau are resolved together by a
 * Rayleigh-Ritz step, tau = 0.005 after this context's BF16X9 or FP32 solve
 * and 0.05 otherwise (the split-precision BF16X3/X6 starts, or vectors from
 * elsewhere).
 * Errors: BDG_EINVAL (n != 2V, null pointers, ldz < n), BDG_ENOMEM,
 * BDG_EUNSUPPORTED (a group of coupled close eigenvalues larger than the
 * cluster step handles), BDG_ENOCONV if tol is not reached within max_iter
 * (the refined pairs are still written and the achieved residual reported). */
int bdg_refine(bdg_ctx *ctx, const bdg_grid *grid, double mu, const double *U,
               const double2 *Delta, int64_t n, double *w, double2 *Z, int64_t ldz,
               int max_iter, double tol, double *resid_out, double *orth_out,
               int *iters_out, cudaStream_t stream);

/* Local densities of Eq. (densities2) over the states with 0 < E_n < Ec:
 *   n(r)  = 2 sum (|v_n|^2 f_T(-E_n) + |u_n|^2 f_T(E_n)),
 *   nu(r) =   sum u_n v_n^* (f_T(-E_n) - f_T(E_n)),
 * with f_T(E) = 1/(1 + exp(E/T)); T = 0 means the step function.
 *   w      device, n ascending eigenvalues; Z device n x n (ldz);
 *   n_out  device, V doubles; nu_out device, V double2.
 * Only the columns j with 0 < w[j] < Ec (a contiguous range, w being sorted)
 * are read from Z.  Accumulation is FP64. */
int bdg_densities(bdg_ctx *ctx, const bdg_grid *grid, int64_t n, const double *w,
                  const double2 *Z, int64_t ldz, double T, double Ec, double *n_out,
                  double2 *nu_out, cudaStream_t stream);

/* Kinetic density and current of Eq. (densities2) over the states with
 * 0 < E_n < Ec:
 *   tau(r) = 2 sum (|grad v_n|^2 f_T(-E_n) + |grad u_n|^2 f_T(E_n)),
 *   j(r)   = 2 sum Im(v_n grad v_n^* f_T(-E_n) - u_n grad u_n^* f_T(E_n)),
 * with the spectral gradient F^-1 (i k) F on the kinetic operator's k set
 * (section "Numerical setup and implementation").  For tau the Nyquist mode
 * k = -pi is kept, so sum_r tau is twice the kinetic energy; for j it has
 * derivative 0, so a real (time-reversal invariant) state carries no current.
 *   w, Z, ldz, T, Ec  as for bdg_densities;
 *   tau_out  device, V doubles;
 *   j_out    device, 3 V doubles: j_x (sites 0..V-1), then j_y, then j_z.
 * Accumulation is FP64.  Errors: BDG_EINVAL (n != 2V, null pointers,
 * ldz < n, T < 0), BDG_ENOMEM. */
int bdg_kinetic_current_densities(bdg_ctx *ctx, const bdg_grid *grid, int64_t n, const double *w,
                                  const double2 *Z, int64_t ldz, double T, double Ec, double *tau_out,
                                  double *j_out, cudaStream_t stream);

/* Allocation-free variant of bdg_densities (no counterpart in the paper; the
 * paper's loop does not constrain allocation).  For callers that must not
 * allocate device memory inside their SCF loop: a host whose own allocator
 * already holds the device memory it may use, or a loop that must not take
 * the implicit device-wide synchronisation of cudaFree.  Same result as
 * bdg_densities; no context, no cudaMalloc/cudaFree, no allocating library
 * routine.  Scratch is one fixed 4 MiB device array per device inside the
 * library, which bounds the grid to V = Nx*Ny*Nz <= 174720 sites; larger
 * grids return BDG_EUNSUPPORTED with a message, before any launch.
 *   grid, n, w, Z, ldz, T, Ec, n_out, nu_out: as for bdg_densities
 *            (caller-owned device buffers, outputs fully overwritten);
 *   stream   a stream of the CURRENT device, on which the call runs;
 *   msg      optional HOST buffer of msg_len bytes for the error text (may
 *            be NULL); set to "" on success.
 * Set-up: the first call on each device looks up the scratch address with
 * cudaGetSymbolAddress (with that device current) and caches it; make that
 * first call before any stream capture.
 * Nothing in the scratch has to start at zero: each word read is written
 * earlier in the same call.  Calls that overlap in time on one device (two
 * streams or two host threads) share the scratch and race: serialise them. */
int bdg_densities_noalloc(const bdg_grid *grid, int64_t n, const double *w,
                          const double2 *Z, int64_t ldz, double T, double Ec,
                          double *n_out, double2 *nu_out, cudaStream_t stream,
                          char *msg, size_t msg_len);

/* Parameters of one self-consistent step (stated substitute functional:
 * contact coupling g with Hartree term, Delta = g nu and U = -g n / 2). */
typedef struct {
    double mu;                /* chemical potential                          */
    double g;                 /* coupling constant (> 0)                     */
    double alpha;             /* linear mixing weight in (0, 1]              */
    double T;                 /* temperature (0: step occupation)            */
    double Ec;                /* energy cutoff (pi^2/2 on the unit grid)     */
    int prec;                 /* BDG_PREC_* for the eigensolve               */
    int refine_iters;         /* max refinement iterations (reduced modes)  */
    double refine_tol;        /* refinement residual target                  */
    const double2 *phase;     /* device, V unit phases e^{i theta} held fixed
                                 (Delta = g Re(nu e^{-i theta}) e^{i theta}),
                                 or NULL for a free phase                     */
    double *n_prev;           /* device, V doubles: density of the previous
                                 step (in) and of this step (out)             */
} bdg_scf_params;

/* The coupling of the stated contact functional (the paper's SLDA functional
 * is not printed: its B and C are deferred to its source code): g > 0 and the
 * uniform Hartree shift U0 that make the uniform state with gap Delta0 at
 * chemical potential mu self-consistent on the grid's spectral k set,
 *   Delta0 = g nu0,  U0 = -g n0 / 2,
 *   n0 = (1/V) sum_{E_k < Ec} (1 - xi_k / E_k),  nu0 = (1/V) sum_{E_k < Ec} Delta0 / (2 E_k),
 *   xi_k = k^2/2 - mu + U0,  E_k = sqrt(xi_k^2 + Delta0^2),  k = 2 pi m / n.
 * Host arithmetic: needs no context and no device.  g_out, U0_out: HOST.
 * Errors: BDG_EINVAL (bad grid, Delta0 <= 0, Ec <= 0, null pointers),
 * BDG_ENOCONV (no Hartree root in [-5000, 0], or no k with E_k < Ec). */
int bdg_gap_coupling(const bdg_grid *grid, double mu, double Delta0, double Ec, double *g_out,
                     double *U0_out);

/* One self-consistent step (paper: the static solution is found
 * "iteratively through a series of diagonalizations"):
 * build H(U, Delta) -> bdg_heev (particle-hole half solve where it applies)
 * -> bdg_refine (modes other than FP64) -> bdg_densities ->
 * U <- (1-alpha) U + alpha (-g n/2), Delta <- (1-alpha) Delta + alpha g nu.
 *   U, Delta  device, V entries each, updated in place;
 *   dn_max_out HOST pointer: max_r |n(r) - n_prev(r)|.  Synchronises. */
int bdg_scf_step(bdg_ctx *ctx, const bdg_grid *grid, const bdg_scf_params *params,
                 double *U, double2 *Delta, double *dn_max_out, cudaStream_t stream);

/* Time evolution of the quasiparticle wavefunctions (paper, Eq. (TDSLDA),
 * "Performance of the Time Evolution Algorithm"):
 *   i d phi_n / dt = H(t) phi_n,  H = [[h, Delta], [Delta^*, -h^*]],  h = T + U - mu,
 * the same H (the operator of Eq. (stHpsi), kinetic T spectral) for every
 * evolved state, with U and Delta given at each instant by the local
 * densities of the evolved states (Eq. (densities2), occupation f_T(E_n) on
 * |u_n|^2 and f_T(-E_n) on |v_n|^2 fixed at the states' initial energies E0)
 * through the stated contact functional  U = U_ext - g n / 2,  Delta = g nu.
 * Stepping: fifth-order Adams-Bashforth-Moulton predictor-corrector with H
 * evaluated twice per step (at the predicted and at the corrected state); the
 * first four steps are classical RK4 steps that build the multistep history
 * (each call starts its own history).  All arithmetic is FP64. */
typedef struct {
    double mu;                /* chemical potential in h                     */
    double g;                 /* contact coupling (U = U_ext - g n/2, Delta = g nu) */
    double T;                 /* temperature of the fixed occupation weights */
    double dt;                /* time step (> 0)                             */
    const double *U_ext;      /* device, V doubles: static external potential,
                                 or NULL for none                            */
} bdg_td_params;

/*   nq       number of evolved states (columns), >= 1;
 *   E0       device, nq doubles: the states' initial energies (occupation
 *            weights);
 *   Psi      device, n x nq double2 (n = 2V, ld ldpsi >= n): the states at
 *            t = 0 on entry, at t = nsteps dt on return (column j = state j,
 *            u rows 0..V-1, v rows V..2V-1 as in bdg_build);
 *   n_out, nu_out  device, V doubles / V double2, or NULL: the densities at
 *            the final time.
 * The context's workspace holds 9 arrays of n x nq double2 (the state, the
 * stage input, two stage results, five history entries).  Errors: BDG_EINVAL
 * (bad grid, nq < 1, ldpsi < n, dt <= 0, nsteps < 0, null pointers),
 * BDG_ENOMEM. */
int bdg_td_evolve(bdg_ctx *ctx, const bdg_grid *grid, const bdg_td_params *params, int64_t nq,
                  const double *E0, double2 *Psi, int64_t ldpsi, int nsteps, double *n_out,
                  double2 *nu_out, cudaStream_t stream);

/* Batched solve of independent Hermitian blocks of uneven sizes (e.g. the kz
 * blocks H_kz = H_perp + (kz^2/2) tau_z of a tube geometry where kz is a good
 * quantum number).  For each block b: A[b] (sizes[b] x sizes[b], lda =
 * sizes[b], destroyed), w[b] (sizes[b] doubles), Z[b] (ldz = sizes[b]).
 *   sizes, A, w, Z  are HOST arrays of nblocks entries (the pointers they hold
 *                   are device pointers);
 *   prec            as for bdg_heev, BDG_HEEV_PH included (every block must
 *                   then be a BdG matrix in the layout of bdg_build).
 * Blocks are solved concurrently by a pool of worker contexts (6 by default,
 * environment BDG_BATCH_WORKERS, 1..16), each with its own workspace, stream
 * and host thread, taking blocks largest first.  The first time a size class
 * with enough blocks is seen, its first blocks are solved with each candidate
 * band width and the fastest is kept in the context for later calls.
 * Ordering: the batch starts after the work queued on `stream`, and `stream`
 * waits for every block.  The call returns on the host once every block's
 * solve has been issued and its status checked (bdg_heev's host decisions).
 * Device memory grows with the number of workers (one workspace each).
 * Errors: BDG_EINVAL (nblocks < 0, null arrays or pointers, a size < 1);
 * otherwise the status of the first block that failed, with its index in
 * the message; blocks not yet started are then skipped. */
int bdg_heev_batched(bdg_ctx *ctx, int nblocks, const int64_t *sizes, double2 *const *A,
                     double *const *w, double2 *const *Z, int prec, cudaStream_t stream);

/* ---- Learned SCF initial guess: a Fourier neural operator --------------
 * No counterpart in the paper's method, which starts its SCF loop from a
 * plain guess or a coarser solution: the network predicts U(r), Re Delta(r),
 * Im Delta(r) from per-site inputs (mu, Delta0, |ansatz|, cos theta,
 * sin theta) so the SCF loop of bdg_scf_step needs fewer iterations; the SCF
 * loop alone decides convergence.
 *   lift P (cin -> width), `layers` Fourier layers
 *     z = W h + b + Re IDFT(R . DFT(h)) on the modes k in [-(modes-1), modes-1]^3,
 *     h' = GELU(z) (no activation after the last layer),
 *   projection Q (width -> cout).
 * Grid: g^3 sites in the site order of bdg_build; activations [batch][site][channel].
 * Parameters: one FP32 vector (layout: P[cin][W], p[W]; per layer W[W][W],
 * b[W], R[M][W][W] complex; Q[W][cout], q[cout]; M = (2 modes - 1)^3); with
 * bf16_weights the kernels use the bf16-rounded weights (FP32 accumulation). */
typedef struct {
    int g;             /* grid points per dimension                      */
    int width;         /* channels of the hidden layers                 */
    int modes;         /* modes kept per dimension: |k| <= modes-1       */
    int layers;        /* Fourier layers                                */
    int cin, cout;     /* input / output channels                       */
    int bf16_weights;  /* 1: bf16-rounded weights, 0: FP32 weights       */
} bdg_fno_config;

/* Host outputs: number of FP32 parameters and FP32 entries of the forward
 * activation cache for a batch. */
int bdg_fno_sizes(const bdg_fno_config *cfg, int batch, int64_t *nparams, int64_t *ncache);
/* out[batch][g^3][cout] = FNO(in[batch][g^3][cin]); cache (device, ncache
 * floats) receives the activations the backward pass needs.  Errors:
 * BDG_EINVAL (bad configuration: 2 modes - 1 must not exceed g). */
int bdg_fno_forward(bdg_ctx *ctx, const bdg_fno_config *cfg, int batch, const float *params,
                    const float *in, float *out, float *cache, cudaStream_t stream);
/* grad (device, nparams floats, overwritten) = d loss / d params given
 * dout = d loss / d out and the cache of the matching forward call. */
int bdg_fno_backward(bdg_ctx *ctx, const bdg_fno_config *cfg, int batch, const float *params,
                     const float *in, const float *cache, const float *dout, float *grad,
                     cudaStream_t stream);
/* Mean squared error over n entries: *loss_out (device float) and
 * dy = 2 (y - target) / n (device). */
int bdg_fno_mse(bdg_ctx *ctx, int64_t n, const float *y, const float *target, float *dy,
                float *loss_out, cudaStream_t stream);
/* One bias-corrected Adam step (Kingma & Ba) on n parameters; m1, m2 device
 * moment buffers (zero before step 1); step >= 1. */
int bdg_fno_adam(bdg_ctx *ctx, int64_t n, float *params, const float *grad, float *m1, float *m2,
                 float lr, float beta1, float beta2, float eps, int step, cudaStream_t stream);

/* Instrumentation (no counterpart in the paper).  With timing enabled, the
 * next bdg_heev / bdg_refine call records a CUDA event on its stream after
 * each internal stage; bdg_stage_times then synchronises on those events and
 * returns, in call order, the stage names (static strings) and durations in
 * milliseconds (each measured from the end of the previous stage).
 *   ms, names  host arrays of max_stages entries (either may be NULL);
 *   count      host: number of stages written. */
int bdg_set_timing(bdg_ctx *ctx, int enable);
/* Cap of every bounded device wait issued through this context and its
 * batched workers: the tensor-core pipeline barriers (tcgen05/TMA) and the
 * stage-2 wait of a sweep on its predecessor.  `cycles` is in SM clock
 * cycles; 0 restores the default (4e9, about 2 s).  A wait that reaches the
 * cap sets the context's error word, the kernel drains the copies and
 * tensor-core operations it has in flight (under the fixed default cap),
 * frees its tensor memory and returns, and the call reports BDG_ETIMEOUT; the
 * next call starts with the error word cleared.  A diagnostic and test knob:
 * a cap of a few cycles makes the waits give up on purpose.  Errors:
 * BDG_EINVAL for cycles < 0. */
int bdg_set_wait_limit(bdg_ctx *ctx, long long cycles);
/* Number of this library's CUDA kernels launched through this context and
 * its batched workers so far (host); every kernel of every path is this
 * library's own. */
int bdg_launch_count(bdg_ctx *ctx, long long *count);
int bdg_stage_times(bdg_ctx *ctx, int max_stages, double *ms, const char **names, int *count);
/* Which path the last calls took (host outputs, either may be NULL):
 * heev_ph = 1 if the last bdg_heev used the particle-hole half solve,
 * refine_ph = 1 if the last bdg_refine used the particle-hole reduction. */
int bdg_last_modes(bdg_ctx *ctx, int *heev_ph, int *refine_ph);

#ifdef __cplusplus
}
#endif

#endif /* BDG_H */
