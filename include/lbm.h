/*
 * lbm.h -- C ABI of the GB300 (sm_103a) implementation of the energy-conserving
 * multiple-relaxation-time finite-difference lattice Boltzmann model for
 * compressible flow of Chen, Xu, Zhang and Li (D2V16; arXiv 0908.3749).
 *
 * The library evolves 16 populations f_i on a 2D grid of nx x ny interior
 * nodes by the paper's Eq. 3,
 *     df_i/dt + v_i . grad f_i = -(M^-1 S_hat (f_hat - f_hat^eq))_i,
 * discretised as in the Appendix (Eq. A.1: forward Euler in time, per-axis
 * Lax-Wendroff in space), with the moment matrix M of Eqs. 5a-5p on the
 * velocity set of Eq. 4 and the equilibria of Eq. 14. Boundary nodes carry the
 * velocity-space equilibrium f^eq = M^-1 f_hat^eq of a boundary state
 * (Sec. V). The gas has R = 1 and gamma = 2: e = rho T + rho |u|^2 / 2.
 *
 * Conventions for every entry point
 *  - Return value: LBM_OK (0) or a negative lbm_status code. No entry point
 *    aborts or throws; lbm_last_error() gives a one-line reason.
 *  - Arrays of fields are row-major [ny][nx] (x fastest), FP64.
 *  - on_device != 0: the pointer is a CUDA device pointer in the current
 *    device's context; otherwise a host pointer. The caller owns every array
 *    it passes and keeps it valid until the call returns.
 *  - Work is issued on the stream given to lbm_create, in order. lbm_step
 *    returns before the GPU finishes; entry points that hand results to the
 *    host (lbm_moments with host output, lbm_audit, lbm_status,
 *    lbm_get_populations with host output) synchronise that stream first.
 *  - The context owns all device memory it allocates (lbm_create) and frees
 *    it in lbm_destroy. A context is used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

/* Status codes. */
enum lbm_status {
  LBM_OK = 0,
  LBM_ERR_INVALID = -1,     /* bad argument or configuration */
  LBM_ERR_UNSUPPORTED = -2, /* valid request the library does not implement */
  LBM_ERR_CUDA = -3,        /* a CUDA call failed (text in lbm_last_error) */
  LBM_ERR_OOM = -4,         /* device allocation failed */
  LBM_ERR_NONFINITE = -5,   /* the state became non-finite or rho <= 0 */
  LBM_ERR_TIMEOUT = -6      /* a bounded device-side wait gave up */
};

/* Storage / arithmetic precision of the populations. */
enum lbm_precision {
  LBM_FP64 = 0,      /* populations and all arithmetic in FP64 */
  LBM_FP32 = 1,      /* populations and transforms in FP32; FP64 for the
                        reported moments (conserved sums, temperature) and
                        the conservation audits */
  LBM_TC_BF16X3 = 2, /* FP32 populations, 16x16 transforms as split-BF16
                        tensor-core products (reserved: LBM_ERR_UNSUPPORTED) */
  LBM_TC_TF32X3 = 3, /* FP32 populations; m = M f and the back-map M^-1 as
                        3xTF32 tensor-core products (tcgen05, FP32
                        accumulation) over 32 x 8 node tiles; equilibria,
                        Lax-Wendroff update, moments and audits as LBM_FP32.
                        Rows y and y + 4 of a tile share an MMA row: a
                        non-finite population of one makes the other's
                        update non-finite in the same step (the watchdog
                        reports that step either way).
                        Grids with 16 x pitch x ny >= 2^32 elements are
                        LBM_ERR_UNSUPPORTED. */
  LBM_DF64 = 4,      /* double-word: each population stored as the
                        unevaluated sum h + l of two FP32 numbers (8 bytes,
                        about 48 significant bits) and every operation of
                        the step done on the FP32 units with error-free
                        transformations (TwoSum, FMA-based TwoProd), two nodes
                        per thread in paired f32x2 instructions; rounding
                        error per operation of order 2^-48 of its operands
                        against FP64's 2^-53. Moments and audits in FP64. */
  LBM_FP32_DWMOM = 5 /* LBM_FP32 populations and transforms, with the
                        conserved moments (rho, j_x, j_y, e) formed from the
                        FP32 populations in double-word arithmetic (error-free
                        butterflies), and the Eq. 14 equilibria and the
                        temperature recovery P = e - |j|^2 / (2 rho) taken in
                        double-word from those, rounded to FP32 where they
                        enter the relaxation; the fused audits sum the
                        double-word moments. */
};

/* Boundary kinds (Sec. V). The ghost node outside a side holds
 * f^eq(state) where the state is:
 *  PERIODIC  the interior node on the opposite side (both opposite sides
 *            must be periodic);
 *  EQ        the fixed state bc.rho, bc.u, bc.v, bc.T (Dirichlet);
 *  REFLECT   the adjacent interior node with the velocity component normal
 *            to the side negated (reflecting wall, Sec. V.B.a);
 *  EXTRAP    2 q1 - q2 for q in (rho, u, v, T), q1 the adjacent node and q2
 *            the next one inwards; q1 if that has rho <= 0 or T <= 0
 *            (linear extrapolation, Sec. V.B.a and V.C);
 *  WALL      (rho of the adjacent node, bc.u, bc.v, bc.T): a moving wall at
 *            fixed temperature (Couette flow, Sec. V.D);
 *  OUTFLOW   the adjacent interior node unchanged (zero-gradient, free
 *            outflow; not used in the paper: open sides of 2D Riemann
 *            problems, where linear extrapolation amplifies waves that
 *            cross the side). */
enum lbm_bc_kind {
  LBM_BC_PERIODIC = 0,
  LBM_BC_EQ = 1,
  LBM_BC_REFLECT = 2,
  LBM_BC_EXTRAP = 3,
  LBM_BC_WALL = 4,
  LBM_BC_OUTFLOW = 5
};

typedef struct {
  int kind;              /* lbm_bc_kind */
  double rho, u, v, T;   /* used by LBM_BC_EQ (all four) and LBM_BC_WALL (u, v, T) */
  /* Optional split of the side (0: the whole side is `kind`). With split = 1
   * a ghost node at position s along the side (its cell-centred x on the y
   * sides, y on the x sides) takes `kind` where s <= split0 + split_rate * t
   * and `far_kind` beyond, t = time level x dt of the state being advanced:
   * e.g. the Mach reflection of Sec. V.B.b, whose bottom is the post-shock
   * inflow up to x = 150 dx and reflecting beyond, and whose top switches
   * from inflow to extrapolation at x = g(t) moving with the incident shock.
   * Neither kind may be LBM_BC_PERIODIC; both share the state above. */
  int split;
  int far_kind;          /* lbm_bc_kind beyond the split */
  double split0, split_rate;
} lbm_bc;

typedef struct {
  int nx, ny;            /* interior nodes, >= 1 each */
  double dx, dy, dt;     /* grid spacing and time step, > 0 */
  double s[16];          /* diagonal of S_hat, s_1..s_16 (Eq. 3); s[0..3]
                            act on conserved moments and have no effect */
  int internal_dof;      /* must be 0: the moment set fixes gamma = 2 */
  int precision;         /* lbm_precision */
  lbm_bc bc[4];          /* sides x-, x+, y-, y+ */
  int audit_every;       /* fused conservation audit every k steps; 0 = off */
} lbm_config;

/* Creates a context for one grid: validates cfg and allocates two population
 * buffers (16 x ny x pitch elements each), the audit scratch and the status
 * block on the current CUDA device. cuda_stream is a cudaStream_t or NULL
 * for the legacy default stream (the context then issues its work on a
 * stream of its own that is ordered with the default stream).
 * Validation: LBM_ERR_INVALID for nx or ny < 1, non-positive or non-finite
 * dx, dy, dt, non-finite or negative s, a bad bc kind, periodic on only one
 * of two opposite sides, or a Courant number max|v_i| dt / dx > 1
 * (max|v_i| = 6); LBM_ERR_UNSUPPORTED for internal_dof != 0 or a precision
 * that is not built. On error *out is NULL. */
int lbm_create(const lbm_config* cfg, void* cuda_stream, lbm_ctx** out);

/* Sets the populations to f^eq(rho, u, v, T) at every node (Sec. V: initial
 * populations are the equilibria of the initial fields) and resets the step
 * counter and the status. Arrays [ny][nx] FP64; rho > 0 and T > 0 expected. */
int lbm_set_init(lbm_ctx* ctx, const double* rho, const double* u,
                 const double* v, const double* T, int on_device);

/* Advances nsteps >= 0 time steps (one fused kernel per step: boundary
 * ghosts, moments, Eq. 14 equilibria, relaxation, back-map, Lax-Wendroff
 * update, and the watchdog / audit epilogue). Asynchronous; a non-finite
 * state is reported by lbm_status. Steps are issued as CUDA-graph replays
 * of fixed-length batches plus single launches for the remainder. */
int lbm_step(lbm_ctx* ctx, long long nsteps);

/* Writes rho, u = j_x / rho, v = j_y / rho and T = e / rho - |u|^2 / 2
 * of the current state ([ny][nx] FP64 each; the conserved sums and T are
 * computed in FP64 whatever the storage precision). Any output pointer may
 * be NULL. Host outputs: synchronises the stream. */
int lbm_moments(lbm_ctx* ctx, double* rho, double* u, double* v, double* T,
                int on_device);

/* Frees every resource of ctx (after synchronising its stream). NULL-safe. */
int lbm_destroy(lbm_ctx* ctx);

/* Grid totals (sum rho, sum j_x, sum j_y, sum e) x dx x dy of the current
 * state in FP64, reduced in a fixed order (bitwise reproducible). Host
 * array of 4. Synchronises. */
int lbm_audit(lbm_ctx* ctx, double totals[4]);

/* Copies up to max_entries of the fused audits (oldest first, the last
 * LBM_AUDIT_RING ones kept) into totals[4 * k] and their time levels into
 * steps[k]; *count receives the number copied. Host arrays. Synchronises. */
#define LBM_AUDIT_RING 1024
int lbm_audit_log(lbm_ctx* ctx, double* totals, long long* steps,
                  int max_entries, int* count);

/* Synchronises and reports the watchdog: *first_bad_step = the first time
 * level whose state had a non-finite value or rho <= 0 (-1 if none);
 * *first_negT_step = the first time level with T <= 0 somewhere (-1 if
 * none; the scheme can recover from this). Either pointer may be NULL.
 * Returns LBM_ERR_NONFINITE when first_bad_step >= 0, else LBM_OK. */
int lbm_status(lbm_ctx* ctx, long long* first_bad_step, long long* first_negT_step);

/* Number of steps taken since lbm_set_init / lbm_set_populations. */
long long lbm_step_count(lbm_ctx* ctx);

/* Checkpoint: copies the populations out ([16][ny][nx], x fastest, in the
 * storage precision: double for LBM_FP64; for LBM_DF64 a pair of floats
 * (h, l) per population, value h + l; float otherwise) and the step
 * counter. lbm_set_populations restores both; a restored run continues
 * bitwise identically (the step has no atomics or races). */
int lbm_get_populations(lbm_ctx* ctx, void* f, long long* step, int on_device);
int lbm_set_populations(lbm_ctx* ctx, const void* f, long long step, int on_device);

/* Bytes per population element (8 or 4) of ctx. */
int lbm_element_size(lbm_ctx* ctx);

/* Launch shape of the step (LBM_FP64 / LBM_FP32 / LBM_DF64 / LBM_FP32_DWMOM).
 * The grid is cut into node tiles (32 x 8 nodes in FP32, 32 x 2 in FP64,
 * 32 x 4 in LBM_DF64). With one block per tile each
 * block updates its tile; with fewer blocks each block takes tiles b, b + G,
 * b + 2G, ... (G blocks), copying its next tile into shared memory while it
 * computes the current one. Results do not depend on it (each node's update
 * is the same, audit partials are kept per tile); only the speed does.
 *  lbm_set_step_blocks: 0 = the default, one block per tile; larger values
 *    are capped at the number of tiles. Synchronises; LBM_ERR_UNSUPPORTED
 *    for LBM_TC_TF32X3 (its own persistent grid, 4 CTAs per multiprocessor).
 *  lbm_step_blocks: the current value (-1 for a NULL ctx).
 *  lbm_autotune: times `launches` step launches for each candidate (one
 *    block per tile; 1 .. k blocks per multiprocessor; ceil(tiles / m) blocks
 *    for m = 2 .. 8) and keeps the fastest. The timed launches read the
 *    current populations and write the spare buffer against scratch
 *    counters: the state, the step count, the watchdog and the audit log are
 *    unchanged. Call it after lbm_set_init / lbm_set_populations.
 *    Synchronises; a no-op for LBM_TC_TF32X3. */
int lbm_set_step_blocks(lbm_ctx* ctx, int blocks);
int lbm_step_blocks(lbm_ctx* ctx);
int lbm_autotune(lbm_ctx* ctx, int launches);

/* Time steps per launch of the FP32 step (LBM_FP32 only): 1 (default) or 2.
 * With 2, lbm_step advances two time levels per launch: each block loads its
 * 32 x 8 tile with a halo of two rows and four columns, computes level n + 1
 * on the tile and a one-node ring around it in shared memory (the ring is
 * computed again by the neighbouring tiles), then level n + 2 on the tile,
 * and stores only that (temporal blocking: one read and one write of the
 * populations per two steps). Each node update is the one-step arithmetic
 * (the ring nodes in unpaired FP32, so results can differ from single steps
 * in the last bit); the watchdog checks both levels and audits use the same
 * fixed-order reductions. Odd step counts end with a single step; contexts
 * with audit_every = 1 always take single steps.
 *  lbm_set_fused_steps: LBM_ERR_INVALID for other values,
 *    LBM_ERR_UNSUPPORTED for LBM_FP64 and LBM_TC_TF32X3 contexts.
 *  lbm_fused_steps: the current value (-1 for a NULL ctx). */
int lbm_set_fused_steps(lbm_ctx* ctx, int steps_per_launch);
int lbm_fused_steps(lbm_ctx* ctx);

/* One-line description of the last error on ctx (or of the last lbm_create
 * failure on this thread when ctx is NULL). Never NULL. */
const char* lbm_last_error(lbm_ctx* ctx);

/* Conservation totals without any device allocation. The paper has no
 * counterpart to this entry point; it exists for callers that cannot
 * allocate device memory (an allocator-free embedding, a fully reserved
 * memory pool, a loop that must not allocate): it computes the same totals
 * as lbm_audit -- (sum rho, sum j_x, sum j_y, sum e) x dx x dy in FP64 -- of a
 * population array the caller owns, using a fixed scratch array that the
 * library holds in device global memory (one partial sum per block of 32 x 8
 * nodes, LBM_NOALLOC_MAX_BLOCKS blocks: 128 KiB per device, kept until the
 * process exits).
 *  f         device pointer, populations [16][ny][pitch] (x fastest), FP64
 *            (precision LBM_FP64) or FP32 (LBM_FP32); only x < nx is read
 *  totals    device pointer to 4 doubles, written by the kernel
 *  cuda_stream  the stream to run on (NULL: legacy default stream)
 * Returns LBM_ERR_INVALID for bad arguments or a grid that needs more than
 * LBM_NOALLOC_MAX_BLOCKS blocks (more than ~1.05e6 nodes); the reason is in
 * lbm_audit_noalloc_last_error(). Asynchronous. All calls share the scratch:
 * calls whose kernels overlap on the GPU (different streams or host threads)
 * race and give wrong totals, so issue them one after another in one stream.
 * The first call on a device looks up the scratch's device address (with that
 * device current) and keeps it for the life of the process; make that call
 * before any stream capture that includes this entry point. A reset of the
 * device (cudaDeviceReset, or an embedder that tears down and rebuilds the
 * device's primary context) invalidates the kept address: do not call this
 * entry point on a device after resetting it. */
#define LBM_NOALLOC_MAX_BLOCKS 4096
int lbm_audit_noalloc(const void* f, int precision, int nx, int ny, long long pitch,
                      double dx, double dy, double* totals, void* cuda_stream);
const char* lbm_audit_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
