/*
 * vfpi.h -- C ABI of the GB300 (sm_103a) velocity fixed-point iteration (V-FPI)
 * contact solver of Lee, Lee & Lee, "Large-Dimensional Multibody Dynamics
 * Simulation Using Contact Nodalization and Diagonalization" (arXiv 2201.09212).
 *
 * Problem (eq. lindyn, eq. scc): find v in R^n, lambda in R^{3 n_c} with
 *     A v = b + J_c^T lambda
 * and, per contact m, the Signorini-Coulomb conditions on
 *     u_m = J_{c,m} v + phi_m e_n,   lambda_m = [lambda_n; lambda_t1; lambda_t2].
 * A is SPD, given as 3x3 block-sparse rows (one block row per node, n = 3N).
 * Contacts are nodal (eq. jcnode): J_{c,m} = [.. R_m ..] for an S-contact on
 * node i, [.. R_m .. -R_m ..] for a D-contact between nodes i and j, with the
 * rows of R_m the contact normal and two tangents (global -> contact frame).
 *
 * Method (Alg. 1 with Alg. 2): with a diagonal step matrix W whose three
 * entries are tied on every node in contact (Prop. 3),
 *     v*      = v^l - W (A v^l - b)                         (eq. pgd1)
 *     eta_m   = J_{c,m} v*,  gamma_m = w_i (+ w_j)          (eq. subp, eq. diagonal)
 *     lambda* = -(eta_m + phi_m e_n) / gamma_m,  lambda_m = ProjectFC(lambda*)  (Alg. 2)
 *     v^{l+1} = v* + W J_c^T lambda                         (eq. vup)
 *     theta   = ||v^{l+1} - v^l||,  stop if theta < theta_th or l = l_max   (Alg. 1)
 * ProjectFC is the strict operator (eq. operator): lambda_n = max(lambda*_n, 0),
 * tangential part projected onto the disk of radius mu lambda_n.
 *
 * Conventions for every entry point
 *  - Arrays are in the context's dtype (VFPI_F32 -> float, VFPI_F64 -> double)
 *    unless stated; positions are always double.
 *  - Every array pointer may be host memory (pageable or pinned) or device
 *    memory; the library asks the CUDA runtime which.  Inputs are copied into
 *    library-owned device memory (re-laid out); the caller keeps ownership of
 *    everything it passes and may change or free it once the call returns (a
 *    call given page-locked host input waits for that copy, and with it for
 *    the work already on the stream; under stream capture the copy is a
 *    graph node instead, which reads the buffer at every replay).
 *  - Work is enqueued on the stream given to vfpi_create (NULL = legacy default
 *    stream).  Calls that return host scalars, or write to host arrays,
 *    synchronise that stream; the others are asynchronous.
 *  - Errors are reported by the return status and never abort the process;
 *    vfpi_last_error() returns a message.  VFPI_NOT_CONVERGED is a soft status:
 *    the last iterate is still returned.
 *  - Node order is the caller's throughout; velocities are [3N] (x, y, z per
 *    node), impulses [n_c * 3] in contact order (lambda_n, lambda_t1, lambda_t2).
 */
#ifndef VFPI_H
#define VFPI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vfpi_ctx* vfpi_t;

typedef enum {
  VFPI_OK = 0,
  VFPI_NOT_CONVERGED = 1,        /* l_max reached with theta >= theta_th       */
  VFPI_ERR_INVALID_ARG = -1,     /* bad sizes, indices, pattern or options      */
  VFPI_ERR_NONFINITE = -2,       /* NaN/Inf in the data or in an iterate        */
  VFPI_ERR_CUDA = -3,            /* a CUDA runtime call failed                  */
  VFPI_ERR_OOM = -4,             /* device allocation failed                    */
  VFPI_ERR_TIMEOUT = -5,         /* a bounded device-side wait ran out          */
  VFPI_ERR_CONTACT_OVERLAP = -6, /* a node appears in more than one contact     */
  VFPI_ERR_UNSUPPORTED = -7      /* option not available in this build          */
} vfpi_status;

enum { VFPI_F32 = 0, VFPI_F64 = 1 };
/* Choice of W (Sec. IV.C): Frobenius-norm minimiser, alpha * I, or caller's. */
enum { VFPI_W_FROBENIUS = 0, VFPI_W_SCALAR = 1, VFPI_W_USER = 2 };
/* ProjectFC (eq. operator): strict (normal clamp, then the disk at mu lambda_n;
 * exact SCC, used for all the paper's results but one) or proximal (Euclidean
 * projection onto the cone; the fixed point is the convex contact problem of
 * eq. ccp, Prop. 5, Thm. 2). */
enum { VFPI_OP_STRICT = 0, VFPI_OP_PROXIMAL = 1 };
/* Residual of Alg. 1: ||dv||_2 (paper) or ||dv||_2 / sqrt(n). */
enum { VFPI_NORM_ABS = 0, VFPI_NORM_RMS = 1 };

/* A in 3x3 block-sparse-row form (Sec. V.A stores A sparse; blocks here).
 * row_ptr [n_nodes+1], col_idx [nnzb] strictly increasing per row with the
 * diagonal block present, vals [nnzb * 9] row-major blocks.  The full
 * (symmetric) pattern is given; the solver assumes no symmetry of the values,
 * and offers the symmetric-storage launch shapes only when create or update
 * finds A = A^T bit for bit. */
typedef struct {
  int32_t n_nodes;
  int32_t nnzb;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const void* vals;
} vfpi_bsr;

/* Nodal contacts (eq. jcnode).  node_j[m] = -1 marks an S-contact; node_j may
 * be NULL when every contact is an S-contact.  R [n_c * 9] row-major with rows
 * n, t1, t2 (orthonormal, det +1, checked to 1e-4); mu [n_c] >= 0; phi [n_c]
 * the normal offset of eq. (scc).  Every node may appear in at most one
 * contact (Prop. 3 needs it; else VFPI_ERR_CONTACT_OVERLAP). */
typedef struct {
  int32_t n_c;
  const int32_t* node_i;
  const int32_t* node_j;
  const void* R;
  const void* mu;
  const void* phi;
} vfpi_contacts;

typedef struct {
  int32_t dtype;           /* VFPI_F32 | VFPI_F64                                  */
  int32_t w_mode;          /* VFPI_W_*                                             */
  double alpha;            /* VFPI_W_SCALAR: W = alpha I                            */
  const void* w_user;      /* VFPI_W_USER: [3N], tied on contact nodes              */
  double theta_th;         /* Alg. 1 threshold                                     */
  int32_t l_max;           /* Alg. 1 iteration cap (>= 1)                          */
  int32_t operator_;       /* VFPI_OP_*                                            */
  int32_t residual_norm;   /* VFPI_NORM_*                                          */
  int32_t n_scenes;        /* 0 or 1: one problem; > 1: independent scenes          */
  const int32_t* scene_ptr;/* [n_scenes+1] node offsets of the scenes (batched)     */
  int32_t block_threads;   /* 0 = default; threads per CTA of the solve kernel       */
  int32_t force_path;      /* 0 = auto: CTA-per-scene (2) for several scenes or a
                              scene of at most 64 slices (2,048 nodes), else
                              grid-wide (1); 1 or 2 forces that path; other
                              values: VFPI_ERR_INVALID_ARG                     */
  int32_t kernel_variant;  /* one of VFPI_VARIANT_*: grid path 0..15, 26..29 (threads per
                              CTA, CTAs/SM register budget, prefetch, TMA ring,
                              symmetric storage, symmetric blocks); scene path 0,
                              30 or
                              VFPI_VARIANT_CL_*; with 0 a nonzero block_threads
                              selects that CTA size, unbudgeted                  */
  int32_t grid_ctas;       /* grid path: CTAs of the persistent launch (0 = all that
                              fit, capped at one warp per 32-row slice)              */
  int32_t chebyshev_ls;    /* Chebyshev acceleration (Alg. 3): slow-start index
                              l_s >= 4 (the estimate rho of eq. varrho first
                              exists after iteration 3), or 0 for the plain
                              iteration of Alg. 1                                 */
  double chebyshev_u;      /* Alg. 3 under-relaxation u in (0, 1] (1 = the printed
                              update of eq. chebyup)                               */
  int32_t n_halo;          /* 0, or: this context is one shard of a scene split by
                              rows across processes/GPUs (see "Sharded scene"
                              below); A's columns then index its n_nodes own
                              nodes and n_halo halo nodes owned by other shards  */
  int32_t reserved;
} vfpi_opts;

/* Grid-path kernel variants (threads per CTA / minimum CTAs per SM the register
 * budget is set for / next-chunk register prefetch).  Pick with the tuner in
 * paper_2201_09212_gb300/tune.py or by hand. */
enum {
  VFPI_VARIANT_DEFAULT = 0,      /* 256 threads, 3 CTAs/SM (80 registers)    */
  VFPI_VARIANT_256_4 = 1,
  VFPI_VARIANT_512_2 = 2,
  VFPI_VARIANT_128_8 = 3,
  VFPI_VARIANT_256_2_PF = 4,
  VFPI_VARIANT_128_4_PF = 5,
  VFPI_VARIANT_512_1_PF = 6,
  VFPI_VARIANT_256_2 = 7,
  /* shared-memory staging: each warp streams its chunks through a ring of
   * N stages filled by 1-D bulk copies (TMA) -- threads per CTA / stages */
  VFPI_VARIANT_TMA_256_4 = 8,
  VFPI_VARIANT_TMA_128_4 = 9,
  VFPI_VARIANT_TMA_128_6 = 10,
  VFPI_VARIANT_TMA_64_8 = 11,
  /* Symmetric storage (grid path; needs A = A^T exactly, which create and
   * update check): only the blocks with c >= r are stored in the sliced-ELL
   * layout, and each row's blocks c < r are read back transposed from
   * there (through L2), about 40 % fewer bytes from HBM per sweep.  The
   * entries are summed in the same order, so the iterates are bitwise those
   * of the full storage; if an update makes A unsymmetric the same shape runs
   * on the full storage.  Threads per CTA / CTAs per SM register budget. */
  VFPI_VARIANT_SYM_256_2 = 12,
  VFPI_VARIANT_SYM_256_3 = 13,
  VFPI_VARIANT_SYM_256_4 = 14,
  VFPI_VARIANT_SYM_512_1 = 15,
  /* Scene path (see force_path): shared-memory-resident
   * cluster kernel.  Each CTA copies its share of a scene's matrix into shared
   * memory once per solve (1-D bulk copies) and every sweep reads it there; a
   * scene larger than one CTA's share is split over the CTAs of a
   * thread-block cluster, which meet at the cluster barrier once per sweep;
   * smaller scenes go one per CTA.  Iterates are bitwise those of the
   * CTA-per-scene kernel (variant 0).  Barzilai-Borwein solves run on the
   * CTA-per-scene kernel.  Names: threads per CTA / CTAs per cluster / CTAs
   * per SM (shared memory is split between them). */
  VFPI_VARIANT_CL_256_1_1 = 16,
  VFPI_VARIANT_CL_256_2_1 = 17,
  VFPI_VARIANT_CL_256_4_1 = 18,
  VFPI_VARIANT_CL_256_8_1 = 19,
  VFPI_VARIANT_CL_128_4_2 = 20,
  VFPI_VARIANT_CL_128_8_2 = 21,
  VFPI_VARIANT_CL_256_4_2 = 22,
  VFPI_VARIANT_CL_256_8_2 = 23,
  VFPI_VARIANT_CL_512_8_1 = 24,
  VFPI_VARIANT_CL_128_8_4 = 25,
  /* Grid path again: the TMA ring with two stages per warp (threads per CTA /
   * stages): half the shared memory per warp of VFPI_VARIANT_TMA_256_4, so
   * twice the warps fit -- for mid-size scenes whose sweeps are bounded by
   * each warp's chain of dependent loads rather than by bandwidth.  The ring
   * kernels (8-11, 26, 27) take a forward Alg. 1 solve's stop test one sweep
   * behind, while the next sweep's grid barrier completes, and discard that
   * sweep on a stop (not with Alg. 3 or D-contacts): v, lambda, the
   * iteration count and theta are those of the other kernels. */
  VFPI_VARIANT_TMA_256_2 = 26,
  VFPI_VARIANT_TMA_128_2 = 27,
  /* Symmetric-block storage, when every 3x3 block of A equals its transpose
   * bit for bit (checked whenever A is set; a mass-spring lattice's blocks
   * are): each block streams as its 6 distinct values, 24 + 4 instead of
   * 36 + 4 bytes, rebuilt to the same 9 entries and FMAs, so the iterates are
   * bitwise those of the full storage.  Forward and adjoint solves
   * (Barzilai-Borwein steps read the full storage); if a later vfpi_update
   * makes a block asymmetric, solves fall back to the full storage.  The
   * 6-value copy (24 bytes per stored slot) is built when the variant is
   * chosen.  Grid path: VFPI_VARIANT_DEFAULT's and VFPI_VARIANT_256_2's
   * shapes; scene path: the CTA-per-scene kernel (block_threads picks its
   * size).  VFPI_ERR_INVALID_ARG for a matrix with an asymmetric block. */
  VFPI_VARIANT_B6_256_3 = 28,
  VFPI_VARIANT_B6_256_2 = 29,
  VFPI_VARIANT_B6_SCENES = 30
};

/* Fill *o with the defaults: F32, Frobenius W, theta_th 1e-5, l_max 200,
 * strict operator, absolute norm, one scene. */
void vfpi_default_opts(vfpi_opts* o);

/* Build a solver for A, b, J_c (eq. lindyn, eq. jcnode).  Validates A's pattern
 * (sorted columns, diagonal present, no block between two scenes), finiteness,
 * and the contacts; lays A out for the device; chooses W (Sec. IV.C, once per
 * A, "recycled" as the paper does); sets the warm start to zero.  h is the
 * time step used by vfpi_integrate.  On success *out owns device memory until
 * vfpi_destroy. */
vfpi_status vfpi_create(const vfpi_bsr* A, const void* b, const vfpi_contacts* Jc,
                        double h, const vfpi_opts* o, void* cuda_stream, vfpi_t* out);

/* Replace the values of A (same pattern; W is recomputed), b and/or the
 * contact set (re-validated; W re-tied).  NULL leaves that part unchanged. */
vfpi_status vfpi_update(vfpi_t ctx, const void* A_vals, const void* b, const vfpi_contacts* Jc);

/* Per-time-step inputs without re-validation: b [3N] and/or phi [n_c] (NULL
 * keeps the old value).  Asynchronous for device pointers. */
vfpi_status vfpi_set_rhs(vfpi_t ctx, const void* b, const void* phi);

/* Warm start v^1 [3N] (Sec. V.A, "warm start"); asynchronous for device input. */
vfpi_status vfpi_set_velocity(vfpi_t ctx, const void* v);
/* Current iterate [3N] and the impulses of the last sweep [n_c * 3]. */
vfpi_status vfpi_get_velocity(vfpi_t ctx, void* v);
vfpi_status vfpi_get_lambda(vfpi_t ctx, void* lambda);
/* lambda* = -(eta + phi e_n) / gamma of the last sweep [n_c * 3] (Alg. 2,
 * before ProjectFC): it fixes the active set the adjoint differentiates at. */
vfpi_status vfpi_get_lambda_star(vfpi_t ctx, void* lambda_star);
/* The diagonal of W [3N] (Sec. IV.C). */
vfpi_status vfpi_get_w(vfpi_t ctx, void* w);
/* Per-step friction coefficients mu [n_c] (eq. scc) without re-validation;
 * W does not depend on mu, so nothing else changes. */
vfpi_status vfpi_set_friction(vfpi_t ctx, const void* mu);

/* Exactly one V-FPI sweep (eq. pgd1, subp, Alg. 2, eq. vup) from the current
 * iterate; *theta_out (nullable, synchronises) gets ||v^{l+1} - v^l||. */
vfpi_status vfpi_step(vfpi_t ctx, double* theta_out);

/* Alg. 1 inner loop to theta < theta_th or l = l_max, entirely on the device
 * (no per-iteration host round trip).  v_inout (nullable): warm start in, v_hat
 * out; lambda_out (nullable); iters_out/theta_out (nullable) for one scene,
 * or arrays of n_scenes entries in batched mode.  Returns VFPI_NOT_CONVERGED
 * if some scene hit l_max. */
vfpi_status vfpi_solve(vfpi_t ctx, void* v_inout, void* lambda_out, int32_t* iters_out,
                       double* theta_out);

/* Enqueue the solve from the current iterate without synchronising (CUDA-graph
 * capturable); read the outcome later with vfpi_get_status. */
vfpi_status vfpi_solve_async(vfpi_t ctx);
/* Synchronise and read the last solve's iteration counts and residuals
 * (arrays of n_scenes entries in batched mode; nullable). */
vfpi_status vfpi_get_status(vfpi_t ctx, int32_t* iters_out, double* theta_out);
/* Synchronise and read, per scene, how the last solve or adjoint solve ended
 * (Alg. 1's two exits, plus the failures): VFPI_OK (theta < theta_th),
 * VFPI_NOT_CONVERGED (l = l_max reached first), VFPI_ERR_NONFINITE (a
 * non-finite residual), VFPI_ERR_TIMEOUT (a bounded wait of the launch ran
 * out; set for every scene).  status_out: host array of n_scenes entries
 * (required).  Returns VFPI_OK unless the read itself fails. */
vfpi_status vfpi_get_scene_status(vfpi_t ctx, int32_t* status_out);

/* Adjoint of the converged fixed point v = f(v; b, phi, mu) of Sec. IV,
 * f(v) = v* + W J_c^T ProjectFC(lambda*(v*)), at the active set frozen by
 * lambda_star [n_c * 3] (caller order; NULL = the last forward sweep's).
 * With P' the Jacobian of the strict operator (Lemma 2 gives its slip part,
 * ||d lambda_t / d lambda*_n|| = mu) and S = W J_c^T diag(P'_m / gamma_m) J_c,
 * the adjoint g_bar solves (I - (I - S)(I - W A))^T g_bar = g_v; it is found by
 * the transposed sweep iterated on u = W (I - S^T) g_bar -- the forward sweep
 * with b := g_v and the contact step replaced by the frozen linear map
 * u_i -= (w_i / gamma) R^T P'^T R (u*_i - u*_j) -- with the forward solve's
 * theta_th and l_max unless vfpi_set_adjoint_tolerance gave the adjoint its
 * own stop test, and with Alg. 3 if vfpi_set_adjoint_chebyshev switched it on.  Outputs (nullable): g_b = dL/db [3N] (= u at
 * convergence), g_phi = dL/dphi [n_c] = -(P'^T z)_n / gamma and
 * g_mu = dL/dmu [n_c] = lambda_n t . z_t (slip), z = J_c u*.  Synchronises. */
vfpi_status vfpi_adjoint(vfpi_t ctx, const void* lambda_star, const void* g_v, void* g_b,
                         void* g_phi, void* g_mu, int32_t* iters_out, double* theta_out);

/* State update x_{k+1} = x_k + h v_hat (eq. disc_dyn) in FP64 on the device;
 * x_inout [3N] double. */
vfpi_status vfpi_integrate(vfpi_t ctx, double* x_inout);

/* One time step (eq. disc_dyn) in one call: b [3N] and phi [n_c] as
 * vfpi_set_rhs, warm start v_start [3N] as vfpi_set_velocity, Alg. 1 as
 * vfpi_solve, v_out [3N] = v_hat and lambda_out [3n_c] as vfpi_get_velocity /
 * vfpi_get_lambda, then x_inout [3N] double += h v_hat as vfpi_integrate.
 * Every pointer is nullable (NULL: that input keeps its current value, that
 * output is not written) and may be host or device memory; v_start and v_out
 * may be the same array.  The copies and kernels are queued back to back on
 * the context's stream -- the positions' upload on a side stream, overlapping
 * the solve -- and the call waits once, at the end, so page-locked host
 * arrays may be changed when it returns.  Results are bitwise those of the
 * separate calls.  Returns as vfpi_solve; VFPI_ERR_INVALID_ARG inside a
 * stream capture (the call waits; capture vfpi_solve_async instead),
 * VFPI_ERR_UNSUPPORTED on a shard. */
vfpi_status vfpi_advance(vfpi_t ctx, const void* b, const void* phi, const void* v_start,
                         void* v_out, void* lambda_out, double* x_inout, int32_t* iters_out,
                         double* theta_out);

/* y = A x with the context's A (x, y [3N]); the only super-linear product of
 * the method (Sec. III.F), exposed for residual checks and dynamics harnesses. */
vfpi_status vfpi_matvec(vfpi_t ctx, const void* x, void* y);

/* Change the launch shape of the solve kernels after create (the tuner's
 * knob): kernel_variant as in vfpi_opts (VFPI_ERR_INVALID_ARG for a variant
 * the context's path does not have), grid_ctas (grid path), block_threads
 * for either path.  Synchronises. */
vfpi_status vfpi_configure_launch(vfpi_t ctx, int32_t kernel_variant, int32_t block_threads,
                                  int32_t grid_ctas);

/* Device time in milliseconds of the most recent solve kernel, measured with
 * CUDA events recorded on the context's stream around that launch. */
vfpi_status vfpi_last_kernel_ms(vfpi_t ctx, float* ms);

/* Sizes of the device layout: [0] padded nodes, [1] slices of 32 rows,
 * [2] stored block slots (incl. padding), [3] kernel path (1 grid, 2 CTA per
 * scene), [4] CTAs of the solve launch, [5] threads per CTA, [6] CTAs that can
 * be resident at once, [7] SMs of the device. */
vfpi_status vfpi_get_layout(vfpi_t ctx, int64_t* info8);

/* How the solve kernels read A (no work on the device): info4[0] the storage
 * of the forward Alg. 1 sweep in the current launch shape (Barzilai-Borwein
 * sweeps always read the full blocks) -- 0 the full 3x3 blocks
 * (36 + 4 bytes per block), 1 the symmetric storage (upper blocks, grid
 * path), 2 the symmetric-block storage (6 values per block, 24 + 4 bytes);
 * [1] every stored block is symmetric bit for bit; [2] A is symmetric (grid
 * path); [3] 0.  The iterates are bitwise those of the full storage in every
 * case. */
vfpi_status vfpi_get_storage(vfpi_t ctx, int32_t* info4);

/* Replace theta_th and l_max of Alg. 1 for later solves (and the adjoint). */
vfpi_status vfpi_set_tolerance(vfpi_t ctx, double theta_th, int32_t l_max);

/* Invertible contact model (eq. invt): Gamma_c + Omega_c in place of Gamma_c with
 * Omega_m = omega_m I, omega [n_c] >= 0 in contact order (NULL: all zero).  The
 * fixed point then satisfies the contact conditions for J v + phi e_n +
 * omega lambda, and lambda = ProjectFC(-(J v + phi e_n) / omega) follows from
 * the velocity alone.  Synchronises. */
vfpi_status vfpi_set_regularization(vfpi_t ctx, const void* omega);

/* Anisotropic friction (Sec. III.E): elliptic cones
 * lambda_n^2 >= lambda_t1^2 / mu^2 + lambda_t2^2 / mu2^2 with mu along t1 (the
 * contact's mu) and mu2 [n_c] along t2; the strict operator then projects
 * lambda*_t onto the ellipse at lambda_n, the maximal-dissipation solution of
 * Prop. 6 (a bounded bisection per contact).  NULL restores isotropic cones.
 * Strict operator only; the adjoint of this model is not built
 * (VFPI_ERR_UNSUPPORTED).  Synchronises. */
vfpi_status vfpi_set_anisotropic_friction(vfpi_t ctx, const void* mu2);

/* Barzilai-Borwein step sizes (Sec. IV.C) for later solves: W = alpha_l I with
 * alpha_l = s^T s / s^T z (rule 1), s^T z / z^T z (rule 2) or the two
 * alternating (rule 3: 1 on odd l, 2 on even), s = v^l - v^{l-1},
 * z = A s = (A v^l - b) - (A v^{l-1} - b); alpha_1 = alpha0, and the previous
 * alpha stays when s^T z <= 0.  Each sweep then has two phases around a grid
 * barrier (the residual, then the update).  Rule 0 returns to the context's W.
 * Excludes Chebyshev acceleration.  The adjoint's frozen active set must then
 * be given explicitly (vfpi_adjoint's lambda_star). */
vfpi_status vfpi_set_barzilai_borwein(vfpi_t ctx, int32_t rule, double alpha0);

/* Chebyshev acceleration of later solves (Alg. 3, eq. chebyup, eq. varrho):
 * nu = 1 before the slow start l_s, 2 / (2 - rho^2) at l_s, then
 * 4 / (4 - rho^2 nu); v^{l+1} = nu (u (v** - v^l) + v^l - v^{l-1}) + v^{l-1}
 * with v** the V-FPI step and rho = min(||v^l - v^{l-1}|| / ||v^{l-1} - v^{l-2}||, 1).
 * rho is computed after the stop test of iteration l >= 3 and used from
 * iteration 4 on, so l_s = 0 switches it off, else l_s >= 4 and 0 < u <= 1
 * (VFPI_ERR_INVALID_ARG otherwise).  The fixed point,
 * W and the adjoint are unchanged. */
vfpi_status vfpi_set_chebyshev(vfpi_t ctx, int32_t l_s, double u);

/* The same acceleration (Alg. 3) for the adjoint solve of vfpi_adjoint, set
 * apart from the forward solve's: the adjoint iteration is linear at the
 * frozen active set and has the spectrum of the forward iteration's
 * linearisation, so the semi-iteration applies to it as it stands.  l_s = 0
 * (the default) switches it off; else l_s >= 4 and 0 < u <= 1.  The adjoint's
 * fixed point is unchanged.  There is no counterpart in the paper, which does
 * not differentiate the solve. */
vfpi_status vfpi_set_adjoint_chebyshev(vfpi_t ctx, int32_t l_s, double u);

/* Stop test of the adjoint solves (vfpi_adjoint), set apart from the
 * forward's: stop when theta = ||u^{l+1} - u^l|| < theta_th, or with
 * relative = 1 when theta < theta_th * ||g_v|| (both in the context's norm,
 * per scene), or at l = l_max (>= 1).  The adjoint's load g_v = dL/dv has the
 * loss's scale, which an absolute threshold set for velocities does not know;
 * with the relative test the iterates scale with g_v exactly (a power-of-two
 * factor gives bitwise scaled results).  Until this is called the adjoint uses
 * the forward's theta_th and l_max (absolute).  There is no counterpart in
 * the paper, which does not differentiate the solve. */
vfpi_status vfpi_set_adjoint_tolerance(vfpi_t ctx, double theta_th, int32_t l_max, int32_t relative);

/* ------------------------------------------------------------------------
 * Allocation-free solve.  The paper has no counterpart to this entry point.
 *
 * For callers that cannot call cudaMalloc: code whose device memory is owned by
 * someone else's allocator or memory pool, plug-ins that may not touch the CUDA
 * allocator, and loops that must never block on an allocation.  Everything
 * above allocates device memory in vfpi_create; this call allocates nothing.
 * It solves one small problem straight from the caller's buffers with
 * W = the Frobenius choice (Sec. IV.C) and the strict operator, one CTA on the
 * given stream, and returns the same iterate as vfpi_solve on that problem.
 *
 *  - FP32 only.  A, b, the contact arrays, v_in, v_out and lambda_out
 *    (n_c * 3, caller's contact order) must be device memory; iters_out and
 *    theta_out are host scalars (nullable).  The call synchronises the stream
 *    to read them back.  On the device, before any block is read, the call
 *    checks row_ptr (row_ptr[0] == 0, row_ptr[n_nodes] == A->nnzb, 1..n_nodes
 *    blocks per row) and the node indices of the contacts, then the column
 *    indices; a failure gives VFPI_ERR_INVALID_ARG.  A node claimed by two
 *    contacts, or a D-contact joining a node to itself, gives
 *    VFPI_ERR_CONTACT_OVERLAP.  Nothing else of vfpi_create's validation runs
 *    (sorted columns, finite values, orthonormal frames, mu >= 0 are the
 *    caller's to guarantee).  On any of these errors no output is written.
 *  - Limit: n_nodes <= VFPI_NOALLOC_MAX_NODES (4096, i.e. 12,288 DOF) and
 *    n_c <= n_nodes; larger problems are rejected with VFPI_ERR_INVALID_ARG.
 *  - Its scratch is a fixed array of 68 * VFPI_NOALLOC_MAX_NODES + 64 =
 *    278,592 bytes in device memory, part of the library image: every GPU
 *    that loads the library holds it until the process exits.  The first call on a device looks up the array's device
 *    address (with that device current); make that first call before any
 *    stream capture.
 *  - All calls on a device share that one array, and it keeps the previous
 *    call's contents (the call clears what must start empty).  Calls that
 *    overlap on the GPU -- on different streams, or from different host
 *    threads -- race on it; serialise them.
 * ---------------------------------------------------------------------- */
#define VFPI_NOALLOC_MAX_NODES 4096
vfpi_status vfpi_solve_noalloc(const vfpi_bsr* A, const float* b, const vfpi_contacts* Jc,
                               double theta_th, int32_t l_max, int32_t residual_norm,
                               const float* v_in, float* v_out, float* lambda_out,
                               int32_t* iters_out, double* theta_out, void* cuda_stream);
/* ------------------------------------------------------------------------
 * Sharded scene.  Only the product A v couples nodes (Sec. III.F); the
 * contact step of Alg. 2 is local to a contact's node(s).  So one scene can be
 * split by rows: each shard owns a contiguous range of nodes (on the lattices
 * here, a slab of z-layers), keeps their rows of A, b, W and their contacts,
 * and per sweep needs the latest v of its halo -- the other shards' nodes that
 * its rows reference -- plus the sum of every shard's ||dv||^2 for theta.
 *
 * vfpi_create with opts.n_halo > 0 makes such a shard: A has n_nodes rows (its
 * own nodes); a column index c < n_nodes is own node c, c >= n_nodes is halo
 * node c - n_nodes.  A row's columns need not increase (keep the unsplit
 * scene's order and the row sums are bit for bit those of the unsplit scene)
 * but each appears once, the diagonal block included (so a row holds 1 to
 * n_nodes + n_halo blocks).  A contact joins own nodes, except that one node
 * of a D-contact may be a halo node (a "split" contact: the other shard holds
 * it too, with the roles of the nodes unchanged); an S-contact on a halo node,
 * or a D-contact between two halo nodes, gives VFPI_ERR_INVALID_ARG.  A shard
 * runs on the grid path (full storage), without Barzilai-Borwein steps, the
 * adjoint or vfpi_matvec (VFPI_ERR_UNSUPPORTED).
 *
 * A sweep of the whole scene is then: every shard calls vfpi_shard_sweep; the
 * callers sum the shards' sumsq (theta^2 of Alg. 1 = the sum; rms: / n of the
 * whole scene) and take the stop test; each shard reads the rows its
 * neighbours need with vfpi_get_nodes and sets the rows it receives with
 * vfpi_set_halo.  The package's shard module drives this over
 * torch.distributed (NCCL between GPUs); nothing here communicates.
 *
 * Alg. 3 on a shard (vfpi_set_chebyshev, or opts.chebyshev_ls): a sweep's
 * weight nu (eq. chebyup) depends on the whole scene's residuals (eq.
 * varrho), which only the caller sees, so after each sweep that the stop
 * test does not end every shard is given the scene's theta of that sweep
 * (vfpi_shard_set_theta); vfpi_set_velocity starts the solve again at sweep
 * 1.  Between launches a shard keeps v^{l-1} next to v^l, as Alg. 3 reads it.
 * theta is summed over shards in another order than over one scene's CTAs,
 * so nu, and with it the iterates, agree with the unsplit solve to rounding
 * (bit for bit without Chebyshev).
 *
 * Split contacts.  The step of a D-contact (Alg. 2) needs v* (eq. pgd1) of
 * both nodes, so on a shard with split contacts a sweep has a second half:
 * after vfpi_shard_sweep, the shard gives the v* of its own endpoints
 * (vfpi_get_split_vstar), receives the other endpoints' v* from their shards,
 * and vfpi_finish_split takes each contact's step and eq. (vup) for its own
 * endpoint.  Both shards of a split contact take the step from the same
 * inputs, so both get the same lambda and each node the unsplit solve's
 * v^{l+1}.  The Frobenius-norm W (Sec. IV.C) is tied over a D-contact's two
 * nodes and formed from both nodes' row statistics: before the first sweep
 * (and after vfpi_update), each shard exchanges those of its endpoints
 * (vfpi_get_split_stats, vfpi_set_split_stats).  Split contacts are counted
 * and ordered as the caller's contact list orders them (k = 0..n_split-1);
 * arrays below are indexed by that k.
 * ---------------------------------------------------------------------- */

/* info2[0] = n_halo, info2[1] = n_split (the split contacts). */
vfpi_status vfpi_get_shard_info(vfpi_t ctx, int32_t* info2);
/* After a sweep that does not end the solve: theta (>= 0) of Alg. 1 for the
 * whole scene (sqrt of the shards' summed sumsq, times 1 / sqrt(n) of the
 * whole scene with the rms norm).  The shard's next sweep is the following
 * one; with Alg. 3 its weight nu comes from the recurrence of eq. varrho and
 * eq. chebyup on these thetas.  VFPI_ERR_UNSUPPORTED on a context that is not
 * a shard, VFPI_ERR_NONFINITE for a negative or non-finite theta. */
vfpi_status vfpi_shard_set_theta(vfpi_t ctx, double theta);

/* One sweep (eq. pgd1, Alg. 2, eq. vup) of this shard's rows from its current
 * iterate and the halo values last set; the iterate advances (the own
 * endpoints of split contacts stay at v^l until vfpi_finish_split).
 * sumsq_out (host double, nullable): this shard's FP64 sum of
 * ||v^{l+1} - v^l||^2 over its rows (without the own endpoints of split
 * contacts), in a fixed order.  Synchronises the stream when sumsq_out is set. */
vfpi_status vfpi_shard_sweep(vfpi_t ctx, double* sumsq_out);
/* Copy the current v of own nodes nodes[0..n) (indices < n_nodes, host or
 * device array) into out [3n] (host or device).  An index out of range gives
 * VFPI_ERR_INVALID_ARG and out is not written (a host list is checked on the
 * host and the call does not wait for the GPU when out is device memory; a
 * device list is checked on the device, and the call synchronises). */
vfpi_status vfpi_get_nodes(vfpi_t ctx, const int32_t* nodes, int32_t n, void* out);
/* Set the v of halo nodes [first, first + n) from vals [3n] (host or device);
 * 0 <= first, first + n <= n_halo. */
vfpi_status vfpi_set_halo(vfpi_t ctx, int32_t first, int32_t n, const void* vals);
/* out [6 n_split] (host or device double): for split contact k, the row
 * statistics of its own endpoint -- a_rr of its three DOFs, then ||A_r*||^2 of
 * the three (FP64, the terms of the Frobenius W) -- of the current A. */
vfpi_status vfpi_get_split_stats(vfpi_t ctx, double* out);
/* partner [6 n_split] (host or device double): the other endpoints'
 * statistics, as their shards' vfpi_get_split_stats gave them.  With
 * VFPI_W_FROBENIUS, W is formed again; other W modes do not use them.  Until
 * this call (after vfpi_create, vfpi_update), vfpi_shard_sweep with split
 * contacts and VFPI_W_FROBENIUS gives VFPI_ERR_INVALID_ARG.  Non-finite
 * values give VFPI_ERR_NONFINITE. */
vfpi_status vfpi_set_split_stats(vfpi_t ctx, const double* partner);
/* out [3 n_split] (host or device, the context's dtype): v* of each split
 * contact's own endpoint, from the last vfpi_shard_sweep. */
vfpi_status vfpi_get_split_vstar(vfpi_t ctx, void* out);
/* Second half of a shard sweep: partner_vstar [3 n_split] (host or device,
 * the context's dtype) holds the other endpoints' v*; each split contact's
 * step (Alg. 2 with gamma = w_i + w_j, eq. diagonal) gives lambda and its own
 * endpoint's v^{l+1} (eq. vup).  sumsq_out (host double, nullable): this
 * shard's whole FP64 ||v^{l+1} - v^l||^2 of the sweep (vfpi_shard_sweep's sum,
 * which leaves out the own endpoints of split contacts, plus theirs);
 * synchronises the stream when set and then reports the sweep's outcome as
 * vfpi_shard_sweep does (VFPI_ERR_TIMEOUT, ...).  With no split contacts it
 * only reads the sum, so that a caller can launch several shards' sweeps
 * (vfpi_shard_sweep with sumsq_out NULL) before waiting for any. */
vfpi_status vfpi_finish_split(vfpi_t ctx, const void* partner_vstar, double* sumsq_out);

/* Message for the last failing vfpi_solve_noalloc call of this host thread. */
const char* vfpi_noalloc_last_error(void);

const char* vfpi_last_error(vfpi_t ctx);
const char* vfpi_status_string(vfpi_status s);
void vfpi_destroy(vfpi_t ctx);

#ifdef __cplusplus
}
#endif
#endif /* VFPI_H */
