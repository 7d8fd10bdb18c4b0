/*
 * lbm_batch.h -- C ABI for batches of independent quasi-1D shock tubes advanced
 * by the D2V16 MRT-FD scheme (same method as lbm.h: Eq. 3 with the moment
 * matrix of Eqs. 5a-5p, the Eq. 14 equilibria and the Lax-Wendroff update of
 * Eq. A.1), in one persistent kernel launch per call.
 *
 * A tube is the paper's 1D Riemann problem of Sec. V.A on nx nodes, one node
 * deep with y periodic (so every y-derivative vanishes), its two ends held at
 * the equilibria of the initial left and right states (Sec. V.A: f = f^eq on
 * the boundary nodes). Tubes differ in nx, dx, relaxation rates and states;
 * all share dt. Populations are FP32 (16 x sum(nx) values, SoA); the reported
 * moments, conserved totals and temperatures are computed in FP64.
 *
 * Conventions as in lbm.h: status codes, caller-owned arrays valid for the
 * duration of the call, work on the stream given at creation, synchronising
 * entry points say so. Field arrays are the concatenation of the tubes in
 * order (tube t starts at sum of nx[0..t-1]).
 */
#ifndef LBM_BATCH_H
#define LBM_BATCH_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_batch lbm_batch; /* opaque, library-owned */

typedef struct {
  int ntubes;            /* >= 1 */
  const int* nx;         /* [ntubes] nodes per tube, >= 2, host */
  const double* dx;      /* [ntubes] node spacing, > 0, host */
  double dt;             /* common time step, > 0; 6 dt / dx <= 1 for every tube */
  const double* s;       /* [ntubes][16] relaxation rates s_1..s_16, host */
  const double* left;    /* [ntubes][4] (rho, u, v, T) held at the x- end, host */
  const double* right;   /* [ntubes][4] (rho, u, v, T) held at the x+ end, host */
} lbm_batch_config;

/* Validates cfg, builds the work list (tiles of each tube) and allocates the
 * population buffers and per-tube tables on the current device. */
int lbm_batch_create(const lbm_batch_config* cfg, void* cuda_stream, lbm_batch** out);

/* f = f^eq(rho, u, v, T) at every node; arrays of sum(nx) FP64 values. Resets
 * the step counter and the per-tube status. */
int lbm_batch_set_init(lbm_batch* b, const double* rho, const double* u,
                       const double* v, const double* T, int on_device);

/* Advances every tube by nsteps >= 0 steps in ONE persistent kernel launch
 * (replayed from a CUDA graph captured per distinct nsteps): each resident
 * block processes its share of the tiles, then all blocks meet at a grid
 * barrier before the next step. The barrier's spin is bounded (about 1 s);
 * if it expires the kernel records LBM_ERR_TIMEOUT (see lbm_batch_status)
 * and every block returns. Asynchronous. */
int lbm_batch_step(lbm_batch* b, long long nsteps);

/* rho, u, v, T of every node in FP64 (conserved sums and T recovered in FP64
 * from the FP32 populations). NULL outputs are skipped. Host outputs
 * synchronise. */
int lbm_batch_moments(lbm_batch* b, double* rho, double* u, double* v, double* T,
                      int on_device);

/* Per-tube totals (sum rho, sum j_x, sum j_y, sum e) x dx in FP64, reduced in
 * a fixed order. totals: host [ntubes][4]. Synchronises. */
int lbm_batch_audit(lbm_batch* b, double* totals);

/* Synchronises. first_bad (host [ntubes], may be NULL): first time level at
 * which the tube had a non-finite value or rho <= 0, -1 if none; *nbad: number
 * of such tubes; *timeout: 1 if a grid barrier gave up. Returns
 * LBM_ERR_TIMEOUT if it did, else LBM_OK (unstable tubes are reported, not an
 * error of the batch). */
int lbm_batch_status(lbm_batch* b, long long* first_bad, int* nbad, int* timeout);

/* Tiling: tile = nodes per work item, threads = threads per block; each
 * thread updates node pairs, so tile is 2 or 4 x threads. The pairs built:
 * (128, 64), (256, 64), (256, 128), (512, 128), (512, 256), (1024, 256),
 * (1024, 512), (1024, 128); anything else is LBM_ERR_INVALID. */
int lbm_batch_set_tiling(lbm_batch* b, int tile, int threads);
int lbm_batch_get_tiling(lbm_batch* b, int* tile, int* threads, int* blocks);

/* Autotuner: times every (tile, threads) candidate for `trial_steps` steps on
 * the live GPU (restoring the populations afterwards), keeps the fastest and
 * returns it in chosen[0..1]. When cache_path is not NULL the result is read
 * from / written to that JSON file, keyed by the GPU name and a hash of the
 * tube lengths. Synchronises. */
int lbm_batch_autotune(lbm_batch* b, int trial_steps, const char* cache_path, int* chosen);

/* Test hook for the bounded barrier: block `block` skips its arrival at the
 * barrier after step `step` of the next launch (-1 disables). Used to check
 * that an expired wait is reported as LBM_ERR_TIMEOUT without hanging. */
int lbm_batch_debug_skip_arrival(lbm_batch* b, int block, long long step);

long long lbm_batch_step_count(lbm_batch* b);
int lbm_batch_total_nodes(lbm_batch* b, long long* total);
int lbm_batch_destroy(lbm_batch* b); /* NULL-safe */
const char* lbm_batch_last_error(lbm_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_BATCH_H */
