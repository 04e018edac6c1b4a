/*
 * tdgrad — two-electron term of the TDA-TDDFT nuclear gradient on GB300.
 *
 * C-ABI of libtdgrad.so.  The library evaluates, for a list of density-matrix
 * pairs (A, B, c_J, c_K, c_K_lr, omega),
 *
 *   g[E,x] = sum_pairs sum_{mu nu lam sig, all ordered}
 *              [ c_J   d(mu nu|lam sig)/dE_x    A_{mu nu}  B_{lam sig}
 *              + c_K   d(mu nu|lam sig)/dE_x    A_{mu lam} B_{nu sig}
 *              + c_K_lr d(mu nu|lam sig)_w/dE_x A_{mu lam} B_{nu sig} ],
 *
 * the 4th and 5th terms of the AO-basis excited-state gradient (Sec. II.A,
 * eq. dE_ao) with the two-particle densities Gamma and Gamma^lr of eq. gamma
 * written as pairs: Gamma = (R,R; c_J=2, c_K=-alpha, c_K_lr=-beta) +
 * (P+2P_delta, P; 1/2, -alpha/4, -beta/4).  (|)_w is the erf(omega r)/r
 * operator of eq. lreri_k; d/dE_x follows eqs. deriv and deri (Sec. II.C).
 *
 * Conventions
 *  - Coordinates in bohr, gradient in hartree/bohr.
 *  - Cartesian Gaussian shells (eq. cartG) with l <= 2; components in
 *    lexicographic order (xx, xy, xz, yy, yz, zz).  Contraction coefficients
 *    multiply normalised primitives, and every component carries the x^l
 *    normalisation N_k N_c of its shell.
 *  - Density matrices are nbf x nbf, row-major, in that AO order; they need
 *    not be symmetric.
 *  - All pairs with c_K_lr != 0 and omega > 0 must share one omega
 *    (TG_EUNSUPPORTED otherwise).  omega <= 0 or c_K_lr = 0 drops the lr term;
 *    omega = +inf makes the lr operator equal to 1/r.
 *  - Screening (Sec. II.E, density-multiplied Schwarz bound): a canonical
 *    shell quartet is skipped iff
 *      8 * npair * max(Q'_ab Q_cd, Q_ab Q'_cd) * M_q^2 < screen_tol,
 *    with Q_ab = max_{mu nu} sum_{kl} |c_k c_l| sqrt((k_mu l_nu|k_mu l_nu)),
 *    Q'_ab the same with the primitive mu or nu replaced by its derivative
 *    function (maximised over centre and direction), and M_q the largest of
 *    M(x,y) = max_p sqrt(|c_J|+|c_K|+|c_K_lr|) max(|A_p|,|B_p|) over the shell
 *    blocks ab, cd, ac, ad, bc, bd (both orientations).  screen_tol = 0 keeps
 *    every quartet.
 *  - Shards (rank, nranks): a canonical quartet belongs to a shard iff
 *    max(key(a,b), key(c,d)) mod nranks == rank, key(x,y) = X(X+1)/2 + Y,
 *    X = max(x,y), Y = min(x,y) over shell indices.  Partial gradients of all
 *    shards sum to the full one.
 *
 * Ownership: the caller owns every pointer it passes.  The library copies
 * what it needs during a call and keeps no caller pointer after return; only
 * the opaque handles persist, and they own their device memory.
 * Threading: a handle may be used by one host thread at a time.
 * Errors: every call returns TG_OK (0) or a negative status; on error the
 * output arrays are left untouched.  tg_strerror() names a status.
 */
#ifndef TDGRAD_H
#define TDGRAD_H

#ifdef __cplusplus
extern "C" {
#endif

#define TG_OK 0
#define TG_EINVAL (-1)        /* bad argument (null, size, exponent <= 0 ...) */
#define TG_EUNSUPPORTED (-2)  /* l > 2, more than one lr omega, too many pairs, or a size
                                 beyond int32 indexing: nshell (nshell+1)/2 >= 2^31 shell
                                 pairs, or >= 2^31 primitive pairs kept in one call */
#define TG_ENOMEM (-3)        /* device or host allocation failed (for tests: while the environment
                                 variable TDGRAD_FAIL_ALLOC=1 is set, every growth of the library's
                                 device work areas fails this way, without a CUDA call) */
#define TG_ECUDA (-4)         /* a CUDA runtime call failed */
#define TG_ETIMEOUT (-5)      /* reserved: a bounded device wait expired.  No kernel of this
                                 version waits on another CTA or a flag, so no call returns it. */
#define TG_EROUTER (-6)       /* router missing, malformed or incompatible */

#define TG_FP64 0             /* every primitive quartet in fp64 */
#define TG_MIXED_BOUND 1      /* fp32/fp64 routing by the rigorous bound */
#define TG_MIXED_LEARNED 2    /* fp32/fp64 routing by the learned router */
#define TG_FP32 3             /* every primitive quartet in fp32 (no accuracy target; calibration) */

#define TG_MAX_PAIRS 8

/* Version of this header's structs and calls; tg_abi_version() returns the
 * value the library was built with.  2: named tg_options fields (autotune,
 * kernel_kind, deterministic, class_mask) and the planning and roofline fields
 * of tg_stats. */
#define TG_ABI_VERSION 2

/* tg_options.kernel_kind: which class-kernel form evaluates a class (every
 * form gives the same result to rounding; a form not compiled for a class
 * falls back to the class default) */
#define TG_KERNEL_DEFAULT 0   /* per-class default */
#define TG_KERNEL_THREAD 1    /* one contracted quartet per thread */
#define TG_KERNEL_GROUP 2     /* a group of 32-128 threads per quartet, arrays in shared memory */
#define TG_KERNEL_WARP 3      /* one warp per quartet, every phase spread over its 32 lanes */

typedef struct tg_basis tg_basis;    /* opaque: basis + geometry, device copies */
typedef struct tg_router tg_router;  /* opaque: block router MLP weights */
typedef struct tg_batch tg_batch;    /* opaque: planned multi-molecule evaluation + CUDA graph */

/* One density pair.  A and B are nbf*nbf doubles, row-major; host pointers
 * unless tg_options.device_ptrs is set, then device pointers. */
typedef struct {
    const double *A, *B;
    double c_J, c_K, c_K_lr, omega;
} tg_pair;

typedef struct {
    double screen_tol;      /* density-multiplied Schwarz threshold; default 1e-10 (Sec. II.E) */
    int precision;          /* TG_FP64 (default), TG_MIXED_BOUND, TG_MIXED_LEARNED, TG_FP32.
                               Mixed modes run a tile in fp32 only while the summed error
                               estimate of all fp32 tiles stays below mixed_tol; gradient
                               accumulation and the reduction are always fp64. */
    const tg_router *router;/* required for TG_MIXED_LEARNED */
    double mixed_tol;       /* target max |dg| of the fp32 route, default 1e-6 Ha/bohr */
    int device_ptrs;        /* 1: A, B and grad are device pointers */
    void *stream;           /* cudaStream_t; NULL = legacy default stream */
    int rank, nranks;       /* shard; default 0 / 1 */
    int timing;             /* 1: time every class kernel with CUDA events (tg_stats.class_ms) */
    int autotune;           /* 0 (default): the per-class default kernel forms and grids.
                               tg_batch_create: 1 autotunes every class list (see there).
                               tg_grad2e: 1 tunes every (class, precision) list the same way
                               on the basis's first call with autotune = 1 and reuses the
                               choices on later calls (a list empty at that call keeps the
                               defaults); 2 tunes again on this call.  The tuning launches
                               time sample tiles and do not change the result's definition:
                               every form computes the same quartets in the same precision. */
    int kernel_kind;        /* TG_KERNEL_DEFAULT (default), _THREAD, _GROUP or _WARP */
    int deterministic;      /* 1 (default): fixed-order fp64 sums, bitwise reproducible on one
                               device for one launch configuration.  Every path of this
                               version is deterministic; 0 is accepted and changes nothing. */
    unsigned class_mask;    /* 0 (default): every angular class; otherwise bit qc keeps class qc
                               (0..20, numbered as in tg_stats.class_quartets) and drops the
                               rest, e.g. for per-class checks and timings */
    int shard_mode;         /* TG_SHARD_PAIR_KEY (default) or TG_SHARD_TILES, see below */
    int reserved[3];        /* must be 0 */
} tg_options;

/* tg_options.shard_mode with nranks > 1:
 * TG_SHARD_PAIR_KEY: the quartet shards of the top of this file (pair keys mod nranks).
 * TG_SHARD_TILES: the screened tile list of every angular class, in the planner's order
 *   (decreasing cost), is dealt cyclically BEFORE the fp32 / fp64 split: its tile i
 *   belongs to rank i mod nranks.  The route is the one of the whole call (the mixed_tol
 *   budget covers all ranks' tiles together), and a rank holds the same tiles at every
 *   precision, so its fp32 / mixed partial can be checked against its fp64 partial.  Each
 *   rank runs 1/nranks of every class's tiles (balanced cost, no quartet filter inside the
 *   kernels); the partial gradients of all ranks sum to the full one.  tg_grad2e only. */
#define TG_SHARD_PAIR_KEY 0
#define TG_SHARD_TILES 1

/* The tiles of one class list of ntiles screened tiles that rank evaluates under
 * TG_SHARD_TILES: *count tiles, first, first + stride, ...  Host only. */
int tg_tile_shard(long long ntiles, int rank, int nranks, long long *first, long long *count, long long *stride);

typedef struct {
    double seconds;               /* wall time of the call (host clock) */
    long long quartets;           /* canonical shell quartets evaluated */
    long long prim_quartets;      /* primitive quartets evaluated */
    long long fp32_quartets;      /* quartets routed to fp32 */
    long long pairs;              /* shell pairs kept after pair screening */
    long long tiles;              /* quartet tiles of the call after screening (tg_grad2e:
                                     the whole system's, before a TG_SHARD_TILES shard) */
    int launches;                 /* CUDA kernels launched by the call */
    int grid;                     /* CTAs of each persistent class launch */
    double class_ms[21];          /* per angular class: fp64 kernel time (only with timing = 1) */
    double class_ms_fp32[21];     /* per angular class: fp32 kernel time (only with timing = 1) */
    long long class_quartets[21];            /* angular class qc = P(P+1)/2 + Q, bra pair class
                                                P >= ket pair class Q, pair classes ss ps pp
                                                ds dp dd = 0..5 */
    long long class_prim_quartets[21];       /* fp64 primitive quartets */
    long long class_prim_quartets_fp32[21];  /* fp32 primitive quartets */
    long long class_bra_prims[21];           /* fp64: bra primitive pairs visited (one per
                                                quartet and bra primitive pair) */
    long long class_bra_prims_fp32[21];      /* the same for fp32 */
    double plan_ms;               /* host clock: densities, block factors, pair screening, class
                                     sort, tile list and routing, up to the first class launch */
    double fp64_flop, fp32_flop;  /* algorithmic FLOPs of the evaluated primitive quartets per
                                     precision (the per-class count of the McMurchie-Davidson
                                     evaluation, 2 per FMA) */
    double fp64_frac_peak;        /* with timing = 1: fp64_flop / summed fp64 class-kernel time,
                                     over the device's fp64 FMA peak (SMs x 2 FMA/clk x 2 x clock);
                                     0 otherwise */
    double fp32_frac_peak;        /* the same for fp32 (SMs x 128 FMA/clk x 2 x clock) */
} tg_stats;

/* Fill o with the defaults listed above. */
void tg_options_default(tg_options *o);
/* TG_ABI_VERSION of the built library. */
int tg_abi_version(void);
/* Algorithmic FLOPs of angular class qc (0..20) with nops operators (1: 1/r
 * only, 2: 1/r and erf(omega r)/r) used by tg_stats: per primitive quartet
 * and per bra primitive pair of a quartet.  The count is that of the
 * McMurchie-Davidson evaluation with the density contraction folded into
 * half-transformed Hermite vectors (Sec. II.C, eqs. cartG, deriv, ti): Boys
 * orders, the Hermite R recursion, and each contraction over the index box
 * t <= a_x+b_x, u <= a_y+b_y, v <= a_z+b_z where a function pair's expansion
 * coefficients can be non-zero; an FMA counts 2.  Host only, no device. */
int tg_class_flops(int qc, int nops, double *per_prim_quartet, double *per_bra_prim);

/* Create a basis handle.  xyz_bohr: natom*3; per shell: atom index, l (0..2),
 * primitive count (1..16); exps/coefs: concatenated primitives in shell
 * order, exps > 0.  Uploads the basis and computes the Schwarz factors Q, Q'
 * on the current CUDA device (eq. cartG normalisation, Sec. II.C). */
int tg_basis_create(int natom, const double *xyz_bohr, int nshell, const int *shell_atom,
                    const int *shell_l, const int *shell_nprim, const double *exps,
                    const double *coefs, tg_basis **out);
int tg_basis_nbf(const tg_basis *b);
int tg_basis_natom(const tg_basis *b);
void tg_basis_destroy(tg_basis *b);

/* The two-electron gradient (see the top of this file).  grad: natom*3
 * doubles, overwritten (host unless device_ptrs).  stats may be NULL.
 * npair in 1..TG_MAX_PAIRS.  opt may be NULL (defaults). */
int tg_grad2e(const tg_basis *b, int npair, const tg_pair *pairs, const tg_options *opt,
              double *grad, tg_stats *stats);

/* Spherical shells (Sec. II.C: a shell's 2l+1 spherical functions are a
 * spherical transformation of its Cartesian ones).  The same gradient as
 * tg_grad2e, of the integrals over spherical functions: every A and B of
 * pairs is tg_basis_nsph(b) x tg_basis_nsph(b), row-major, in the spherical
 * AO order -- per shell in shell order: s; p as x, y, z; d as the unit-norm
 * real solid harmonics m = -2 (sqrt3 xy), -1 (sqrt3 yz), 0 (zz - (xx+yy)/2),
 * +1 (sqrt3 xz), +2 ((sqrt3/2)(xx - yy)) of the x^l-normalised Cartesian
 * functions.  The library forms A_cart = T A T^T (T: nbf x nsph, block
 * diagonal over shells) on the device and runs tg_grad2e on them, which
 * gives sum d(mn|ls)_sph A B exactly (linearity).  Options, stats and
 * errors as tg_grad2e (host pointers unless device_ptrs); stats.launches
 * also counts the 2 * npair transforms. */
int tg_basis_nsph(const tg_basis *b);
int tg_grad2e_sph(const tg_basis *b, int npair, const tg_pair *pairs, const tg_options *opt,
                  double *grad, tg_stats *stats);

const char *tg_strerror(int status);

/* ---- Fock-type build (Sec. II.B: the two-electron part of eq. G_2e, the
 * Lagrangian's Fock-type matrices, and of eq. zfock, the Z-vector's; the XC
 * kernel term of those equations is not part of it)
 *
 *   F[mu nu] = sum_p sum_{lam sig} B_p[lam sig] ( c_J (mu nu|lam sig)
 *              + c_K (mu lam|nu sig) + c_K_lr (mu lam|nu sig)_omega )
 *
 * over npair (1..TG_MAX_PAIRS) density matrices B_p (nbf x nbf row-major,
 * need not be symmetric; host pointers unless opt->device_ptrs).  Eq. G_2e
 * is the pair (P~_delta^T; c_J = 2, c_K = -alpha, c_K_lr = -beta); eq. zfock
 * is the two pairs (B^T; 4, -alpha, -beta) and (B; 0, -alpha, -beta).
 * F: nbf*nbf doubles, overwritten.  Screening: a canonical shell quartet is
 * skipped iff 8 * Q_ab Q_cd * M_q < screen_tol, with Q the Schwarz factors of
 * tg_grad2e and M_q the largest over the blocks ab, cd, ac, ad, bc, bd (both
 * orientations) of max(|S_J|, |B_K|, |B_lr|), S_J = sum_p c_J (B_p + B_p^T),
 * B_K = sum_p c_K B_p, B_lr = sum_p c_K_lr B_p (omega > 0); screen_tol = 0
 * keeps every quartet.  fp64 throughout (opt->precision must be TG_FP64);
 * contributions are summed into F with fp64 atomics, so the last bits may
 * change from run to run (opt->deterministic does not apply).  stats may be
 * NULL (quartets, prim_quartets, class counts, timings as in tg_grad2e). */
typedef struct {
    const double *B;
    double c_J, c_K, c_K_lr, omega;
} tg_fpair;
int tg_fock2e(const tg_basis *b, int npair, const tg_fpair *pairs, const tg_options *opt, double *F,
              tg_stats *stats);

/* ---- batched evaluation (many independent molecules, plan once, replay)
 * tg_batch_create plans every molecule (screening, class sort, routing as in
 * tg_grad2e) and captures one CUDA graph whose persistent class launches
 * each cover the tiles of all molecules.  The bases must be distinct handles
 * (a basis holds one plan at a time) and must outlive the batch; with
 * device_ptrs the densities are read from the caller's device buffers at
 * every run (their contents may change, the plan does not), otherwise they
 * are copied at creation.  opt->autotune = 1 autotunes every class list
 * on a sample of 2 to 4 x (SM count) of its tiles taken at a fixed stride
 * over the whole list: the kernel form (thread, group or
 * warp), the persistent grid (1, 2 or 4 CTAs per SM) and the work-unit shape
 * (bra primitive splits per tile: automatic, 1 or 4), searched one
 * coordinate at a time (form, then grid, then splits; 7 timed launches per
 * list), keeping the fastest.
 * tg_batch_run replays the graph on opt->stream and writes grads[m]
 * (natom_m * 3, host unless device_ptrs).  Not part of the paper, which
 * evaluates one system at a time (Sec. II.C). */
int tg_batch_create(int nmol, const tg_basis *const *bases, const int *npair, const tg_pair *const *pairs,
                    const tg_options *opt, tg_batch **out);
int tg_batch_run(tg_batch *batch, double *const *grads, const tg_options *opt, tg_stats *stats);
void tg_batch_destroy(tg_batch *batch);

/* ---- learned block router (fp32 / fp64 routing only; it never skips work)
 * A 16-32-32-1 tanh perceptron maps 16 features of a quartet tile (angular
 * class, log10 of the tile's Schwarz x density bound, of Q and Q' on each
 * side, of the cross and pair density factors, pair-centre distances, pair
 * extents, smallest exponent sums, primitive-pair counts) to the log10 of the
 * tile's largest contribution to one gradient component.  Mixed modes route
 * tiles to fp32 in increasing order of their error estimate e_t while
 * sum e_t^2 <= mixed_tol^2 (independent rounding errors add in quadrature;
 * tg_grad2e takes the tiles bin by bin, 8 bins per factor of 2 in e_t, each
 * tile counted at its bin's upper edge): e_t = eps_rel * 10^(prediction +
 * margin) for TG_MIXED_LEARNED, whose margin is calibrated on measured
 * errors against the fp64 path, and 3e-6 * 128 * nfq * bound for
 * TG_MIXED_BOUND.
 * The paper has no counterpart: its kernels are fp64 throughout (Sec. II.C,
 * II.E). */

/* Per-tile training data: every stride-th screened tile (at most cap) of the
 * call's workload is evaluated in fp64 and in fp32 without reduction.
 * features: cap*16; target: log10 of the tile's largest contribution to one
 * gradient component (its quartets summed per atom and direction, fp64);
 * err32: log10 of the largest |fp32 - fp64| difference of those sums;
 * *n_out: tiles written. */
int tg_tile_samples(const tg_basis *b, int npair, const tg_pair *pairs, const tg_options *opt, int stride, int cap,
                    float *features, float *target, float *err32, int *n_out);

int tg_router_nparam(void);                         /* 1633 */
int tg_router_create(unsigned long long seed, tg_router **out);  /* Xavier-uniform init */
void tg_router_destroy(tg_router *r);
/* params: tg_router_nparam() floats (W1[32][16], b1, W2[32][32], b2, w3[32], b3);
 * mu, sd: 16 feature means / standard deviations; calib: {margin, eps_rel, trained}.
 * Any pointer may be NULL.  tg_router_set returns TG_EINVAL, changing nothing,
 * when a value is not finite, an sd is <= 0 or eps_rel < 0. */
int tg_router_get(const tg_router *r, float *params, float *mu, float *sd, float *calib);
int tg_router_set(tg_router *r, const float *params, const float *mu, const float *sd, const float *calib);
/* GPU training: standardise the features, then `epochs` full-batch Adam steps
 * on the expectile loss mean(w r^2), r = y - yhat, w = q if r > 0 else 1-q.
 * X: n*16 host floats, y: n; loss_hist (nullable): epochs floats. */
int tg_router_train(tg_router *r, int n, const float *X, const float *y, int epochs, float lr, float q,
                    float *loss_hist);
/* Loss and gradient (tg_router_nparam() floats) of the current parameters. */
int tg_router_loss_grad(const tg_router *r, int n, const float *X, const float *y, float q, float *loss,
                        float *grad);
int tg_router_predict(const tg_router *r, int n, const float *X, float *out);

/* Allocation-free loss and gradient of router parameters, for callers that
 * cannot call cudaMalloc or cudaFree where they need it: code running while
 * a stream is captured into a CUDA graph (allocation calls are illegal in a
 * global-mode capture), code sharing the device with a framework whose
 * caching allocator holds the free memory, and latency-critical loops that
 * cannot take the device synchronisation cudaFree may cause.  The paper has
 * no counterpart.
 * Every argument is a caller-owned DEVICE pointer on the current device: X
 * (n*16 standardised-or-raw features), y (n), mu and sd (16 each), params
 * (tg_router_nparam() floats, layout of tg_router_get), loss (1 float) and
 * grad (tg_router_nparam() floats) receive the expectile loss (quantile q)
 * and its gradient, as tg_router_loss_grad computes them.  stream: a
 * cudaStream_t or NULL; the call is asynchronous on it.
 * Scratch: a fixed 3.3 MB device array inside the library (per-block partial
 * sums for n <= 65536; larger n returns TG_EUNSUPPORTED).  Every device that
 * loads the library holds it until the process exits.  All calls on a device
 * share it: calls that overlap on the GPU (different streams, or another
 * host thread) race and must be serialised by the caller.  Every call
 * rewrites the parts it reads, so nothing carries over between calls.
 * The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress) and sets the kernel's shared-memory limit; make that
 * first call before any stream capture. */
int tg_router_loss_grad_noalloc(int n, const float *X, const float *y, const float *mu, const float *sd,
                                const float *params, float q, float *loss, float *grad, void *stream);
/* Router file: int32 {0x54524754 ("TGRT"), version 1, 16, 32}, then the
 * parameters, mu, sd and {margin, eps_rel, trained} as float32, in the host's
 * byte order.  tg_router_load returns TG_EROUTER (and *out = NULL) for a
 * missing, short or foreign file, or one holding non-finite values or an
 * sd <= 0. */
int tg_router_save(const tg_router *r, const char *path);
int tg_router_load(const char *path, tg_router **out);

#ifdef __cplusplus
}
#endif
#endif
