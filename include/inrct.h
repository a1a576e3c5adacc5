/*
 * inrct.h -- C ABI of the GB300-native memory-efficient INR gradient for CT.
 *
 * The library computes, on one GPU, the stochastic gradient of an implicit
 * neural representation (INR) fitted to CT data, following "Memory-efficient
 * optimization of implicit neural representations for CT reconstruction"
 * (arXiv 2604.09884):
 *
 *   min_theta L(P E{f_theta}, y)                         (Sec. 2, Eq. 1)
 *   z = P E{f_theta},  v = P^T dL/dz                     (Sec. 3; Algorithm 1)
 *   g = (n/|I|) sum_{i in I} v_i grad_theta f_theta(x_i)  (Sec. 3, Eq. 2; Algorithm 1)
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every pointer argument to a call (image, sinogram, theta, indices,
 *   gradients, workspace) is DEVICE memory owned by the caller, unless the
 *   argument's comment says "host".  The library never allocates, frees or
 *   keeps a pointer after a call returns.  Descriptor structs are host memory
 *   and are read during the call only.
 * - Calls are asynchronous on the given stream and return a status code.
 *   A non-zero status means nothing was launched (argument errors) or a CUDA
 *   launch failed; inrct_last_error() then returns a message for the calling
 *   thread.  Status codes: see INRCT_OK..INRCT_ERR_TIMEOUT.
 * - Grid: N^d pixels/voxels with centres c_k = -1 + (k + 1/2)(2/N) on
 *   [-1, 1]^d; flat index i = ((iz*N) + iy)*N + ix (x fastest).
 * - Sinogram layout: 2-D [view][bin]; 3-D [view][row v][column u].
 * - theta layout: for every layer in order, W row-major [out][in] then b[out].
 *   FFN: Linear(2F -> w) + ReLU, (n_hidden - 1) x [Linear(w -> w) + ReLU],
 *   Linear(w -> 1).  SIREN: sin(omega0 (W x + b)) layers, same count, then
 *   Linear(w -> 1).
 * - Scratch memory is passed as (ws, ws_bytes); each call documents how to
 *   size it.  Workspace contents need not be initialised.  project,
 *   backproject and grad_step keep the geometry's ray tables in their
 *   workspace between calls: a later call with the same geometry and the same
 *   ws reuses them when the fingerprints written at both ends of the table
 *   region after a completed build still match, and rebuilds them otherwise.
 *   A caller that writes into a workspace between calls must not leave both
 *   fingerprints intact (clearing any byte of either suffices; reusing the
 *   memory for other data normally does).
 */
#ifndef INRCT_H
#define INRCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cudaStream_t;

/* status codes */
#define INRCT_OK 0
#define INRCT_ERR_INVALID_ARG 1
#define INRCT_ERR_UNSUPPORTED 2
#define INRCT_ERR_WORKSPACE 3
#define INRCT_ERR_CUDA 4
#define INRCT_ERR_TIMEOUT 5

/* geometry kinds */
#define INRCT_PAR2D 0  /* 2-D parallel beam */
#define INRCT_FAN2D 1  /* 2-D fan beam, equiangular (curved) detector */
#define INRCT_CONE3D 2 /* 3-D circular cone beam, flat panel */

/* INR kinds and arithmetic of the MLP */
#define INRCT_FFN_RELU 0 /* Gaussian Fourier features + ReLU MLP */
#define INRCT_SIREN 1    /* sine-activated MLP */
#define INRCT_HASH 2     /* multiresolution hash encoding + ReLU MLP (FP32 path only) */
#define INRCT_FP32 0     /* SIMT FP32 path (the plain comparator) */
#define INRCT_BF16 1     /* tcgen05 BF16 x BF16 -> FP32 tensor-core path */

/* loss kinds */
#define INRCT_LOSS_LS 0  /* 1/2 ||z - y||^2, dL/dz = z - y (Sec. 2) */
#define INRCT_LOSS_FLS 1 /* 1/2 (z-y)^T F (z-y), dL/dz = F (z - y), F = ramp filter (Sec. 2) */

/*
 * Scan geometry (the discrete projector P of Sec. 3; the paper does not fix a
 * projector model, this library implements Joseph's ray-driven interpolation).
 * Lengths are in pixel units at the isocentre, angles in radians.
 *   view angle k:  angle0 + angle_span * k / n_views
 *   PAR2D:  bin b lies at (b - (n_bins_u-1)/2) * du pixels from the centre.
 *   FAN2D:  source at distance sod; fan angle of bin b is (b - (n_bins_u-1)/2) * du / sod.
 *   CONE3D: source at distance sod, flat panel at distance sdd from the source,
 *           pitches du, dv measured at the isocentre; n_bins_v rows.
 */
typedef struct {
  int kind;
  int n_views;
  int n_bins_u;
  int n_bins_v; /* 1 for 2-D */
  double du, dv;
  double sod, sdd;
  double angle0, angle_span;
} inrct_geom;

/*
 * Grid: d in {2, 3}, N pixels per side, flat index row-major with x fastest.
 * fov selects the grid points the method samples (Sec. 3 samples the INR inside
 * a field-of-view mask and does not give its shape): 0 = every grid point, 1 =
 * the inscribed disk (2-D) or the cylinder along z (3-D), i.e. the points with
 * (2 k_x + 1 - N)^2 + (2 k_y + 1 - N)^2 <= N^2 (an exact integer test).  With
 * fov = 1 inr_eval_grid writes 0 outside the mask, and listed points outside it
 * contribute nothing to inr_weighted_vjp (as out-of-range indices do); the
 * projector is unaffected.  A zero-initialised descriptor means fov = 0.
 */
typedef struct {
  int d;
  int N;
  int fov;
} inrct_grid;

/*
 * INR architecture (Sec. 4 trains FFN, SIREN and hash-encoded MLPs; all three
 * are implemented).  B: device pointer, n_feat x d FP32 row-major Fourier
 * matrix (FFN only; may be NULL otherwise).  The FFN input is
 * [cos(2 pi B x); sin(2 pi B x)] (cos block first).
 *
 * Hash encoding (INRCT_HASH; the paper names the encoding of Mueller et al.
 * without parameters, so these are the usual ones): level l = 0..hash_levels-1
 * has resolution N_l = floor(hash_base * hash_growth^l), computed on the host
 * in double precision.  Grid point with integer index k (per axis) has level
 * coordinate (2k + 1) N_l / (2N); its 2^d surrounding vertices c (integers in
 * [0, N_l]) index the level's table of T = 2^hash_log2_T entries densely
 * (sum_k c_k (N_l + 1)^k) when (N_l + 1)^d <= T, else by the spatial hash
 * (c_0 * 1) xor (c_1 * 2654435761) xor (c_2 * 805459861) in 32-bit unsigned
 * arithmetic, modulo T.  The level's hash_feats features are the multilinear
 * interpolation of the vertices' entries; the MLP input is the concatenation
 * over levels (level-major), followed by n_hidden Linear + ReLU layers and
 * Linear(width, 1).  theta then begins with the tables, FP32
 * [level][entry][feature], before the layers, and must be 8-byte aligned
 * (INRCT_ERR_INVALID_ARG otherwise).  The table gradient is a scatter-add
 * with FP64 atomics, so its last bits may differ between runs.
 */
typedef struct {
  int kind;    /* INRCT_FFN_RELU, INRCT_SIREN or INRCT_HASH */
  int d;       /* input dimension, equals the grid's */
  int n_feat;  /* F, FFN only */
  const float* B;
  float omega0; /* SIREN only */
  int n_hidden; /* number of nonlinear layers */
  int width;    /* hidden width */
  int prec;     /* INRCT_FP32 or INRCT_BF16 (hash: INRCT_FP32 only) */
  /* hash encoding, INRCT_HASH only (zero otherwise) */
  int hash_levels;    /* 1..16 */
  int hash_feats;     /* features per level: 1, 2, 4 or 8; hash_levels * hash_feats <= 64 */
  int hash_log2_T;    /* table size 2^hash_log2_T entries per level, 4..24 */
  int hash_base;      /* coarsest resolution N_0, 1..65536 */
  double hash_growth; /* per-level growth factor, 1 <= hash_growth <= 4, N_l <= 2^20 */
  /* Optional host copy of B (the same F x d values, row-major), or NULL; FFN only.  With it,
   * the BF16 grid evaluation of a Fourier-feature network with F <= 1024 passes the features'
   * coefficients to its kernel as launch parameters, read through the constant cache, instead
   * of staging them in shared memory, whose bandwidth the tensor cores' operand reads share
   * (501^3 evaluation of the 512-feature network: 118.5 -> 116.2 ms).  Results are identical
   * either way.  Read during the call only; it must hold the values B holds. */
  const float* B_host;
} inrct_mlp;

/* Adam hyper-parameters (Sec. 4 trains with Adam; Kingma-Ba with bias correction); t is
 * the 1-based index of the step being taken.  Both bias corrections are folded into the step
 * size and epsilon in FP64; theta, m and s are then updated in FP32 with beta1 and beta2 taken
 * as FP32 values. */
typedef struct {
  double lr, beta1, beta2, eps;
  int64_t t;
} inrct_adam;

/* ------------------------------------------------------------------------ */

/* Message for the last failing call on this thread ("" if none). */
const char* inrct_last_error(void);

/* Number of parameters p of an MLP descriptor (0 if invalid). */
int64_t inrct_num_params(const inrct_mlp* mlp);

/* Number of rays m = views x rows x bins (0 if invalid). */
int64_t inrct_num_rays(const inrct_geom* geom);

/* ------------------------------------------------------------------------ */
/*
 * project -- z = P x (Sec. 3; Algorithm 1, evaluated without gradient tracking).
 *   image[n] FP32 in, sino[m] FP32 out (overwritten).
 *   Optional loss epilogue (Sec. 2, LS loss): if y != NULL, also writes
 *   resid[m] = z - y and loss_out[0] = 1/2 sum (z - y)^2 (one FP64 device
 *   scalar, overwritten); resid and loss_out may be NULL when y is NULL.
 *   ws: at least inrct_project_ws_bytes(geom, grid) bytes.
 */
size_t inrct_project_ws_bytes(const inrct_geom* geom, const inrct_grid* grid);
int project(const inrct_geom* geom, const inrct_grid* grid, const float* image, float* sino,
            const float* y, float* resid, double* loss_out, void* ws, size_t ws_bytes,
            cudaStream_t stream);

/*
 * project_noalloc -- the same projection and optional LS-loss epilogue as
 * project(), for callers that cannot allocate device memory: for example an
 * application whose device memory belongs to another framework's pool
 * allocator, or a scanner-side loop that reserves all memory at start-up and
 * may not allocate afterwards.  The paper has no counterpart; this is a
 * calling convention of this library only.
 *   The scratch lives in one static device array of INRCT_NOALLOC_SCRATCH_BYTES
 *   bytes inside the library, which every GPU that loads the library keeps
 *   until the process exits.  The call allocates nothing: the caller passes
 *   image, sino (and y, resid, loss_out) exactly as for project().
 *   A geometry whose scratch (inrct_project_ws_bytes) exceeds the array is
 *   rejected with INRCT_ERR_WORKSPACE before anything is launched (2-D
 *   geometries up to about 1400^2 pixels fit; most 3-D ones do not).
 *   Every call made outside stream capture looks up the array's device address
 *   on the device that is current at the call; a call made during stream
 *   capture uses the address found by an earlier call on that device, so make
 *   the first call on a device before any stream capture (otherwise
 *   INRCT_ERR_INVALID_ARG).  All calls on a device share the one array: calls
 *   whose work overlaps on the GPU (different streams, or host threads
 *   without ordering) race on it and must be serialised by the caller.  The
 *   array keeps the last call's contents.  A call reuses the ray tables an
 *   earlier call left there only if they were completely built for the same
 *   geometry (a fingerprint written after the build, checked on the device);
 *   everything else it reads it writes first, so no clearing is needed.
 */
#define INRCT_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int project_noalloc(const inrct_geom* geom, const inrct_grid* grid, const float* image, float* sino,
                    const float* y, float* resid, double* loss_out, cudaStream_t stream);

/*
 * backproject -- v = P^T r (Sec. 3; Algorithm 1), the exact
 * adjoint of project (same interpolation weights), in gather form: every
 * pixel sums its own contributions, so the result is deterministic.
 *   sino[m] FP32 in, image[n] FP32 out (overwritten, not accumulated).
 *   ws: at least inrct_backproject_ws_bytes(geom, grid) bytes.
 */
size_t inrct_backproject_ws_bytes(const inrct_geom* geom, const inrct_grid* grid);
int backproject(const inrct_geom* geom, const inrct_grid* grid, const float* sino, float* image,
                void* ws, size_t ws_bytes, cudaStream_t stream);

/*
 * ramp_filter -- out = F r and loss_out[0] = 1/2 r^T F r for the filtered
 * least-squares loss (Sec. 2: L_FLS = 1/2 (z-y)^T F (z-y), F a ramp filter
 * along the detector rows; Sec. 3: dL/dz = F (z - y)).  F convolves every
 * detector row (one view; one detector row v for the cone) along the bin axis
 * with the Ram-Lak kernel sampled at tau = du * 2/N:
 * (F r)_b = tau sum_k h[k] r_{b-k}, h[0] = 1/(4 tau^2), h[odd k] = -1/(pi^2 k^2 tau^2),
 * h[even k != 0] = 0, zero outside the detector.
 *   r[m] FP32 in, out[m] FP32 out (must not alias r), loss_out one FP64 device
 *   scalar.  At most 6144 bins per row.  ws: inrct_ramp_ws_bytes(geom, grid).
 */
size_t inrct_ramp_ws_bytes(const inrct_geom* geom, const inrct_grid* grid);
int ramp_filter(const inrct_geom* geom, const inrct_grid* grid, const float* r, float* out,
                double* loss_out, void* ws, size_t ws_bytes, cudaStream_t stream);

/*
 * inr_eval_grid -- E{f_theta} = [f(x_1) .. f(x_n)] on the full grid (Sec. 3).
 *   theta[p] FP32 in; image[n] FP32 out.  mlp->prec picks the FP32 SIMT or the
 *   BF16 tcgen05 path.  ws: at least inrct_eval_ws_bytes(mlp, grid) bytes.
 */
size_t inrct_eval_ws_bytes(const inrct_mlp* mlp, const inrct_grid* grid);
int inr_eval_grid(const inrct_mlp* mlp, const float* theta, const inrct_grid* grid, float* image,
                  void* ws, size_t ws_bytes, cudaStream_t stream);

/*
 * inr_weighted_vjp -- scale * sum_{k < n_idx} v[idx[k]] grad_theta f(x_{idx[k]})
 * (Sec. 3, Eq. 2 with scale = n/|I|; equivalently the gradient of the virtual
 * loss of Eq. 3).  Activations are recomputed for the listed points only, so
 * scratch grows with n_idx, never with the grid.
 *   idx[n_idx] int32 flat grid indices (any order, repeats allowed), each in
 *   [0, n); an index outside [0, n) contributes nothing (it is not checked on
 *   the host, which would need a device-to-host copy).  v[n] FP32 (the
 *   backprojected residual on the whole grid).
 *   grad_f64[p] FP64 out (overwritten); grad_f32[p] FP32 out, may be NULL.
 *   ws: at least inrct_vjp_ws_bytes(mlp, grid, n_idx) bytes.
 *   n_idx = 0 is INRCT_ERR_INVALID_ARG.
 */
size_t inrct_vjp_ws_bytes(const inrct_mlp* mlp, const inrct_grid* grid, int64_t n_idx);
int inr_weighted_vjp(const inrct_mlp* mlp, const float* theta, const inrct_grid* grid,
                     const int32_t* idx, int64_t n_idx, const float* v, double scale,
                     double* grad_f64, float* grad_f32, void* ws, size_t ws_bytes,
                     cudaStream_t stream);

/*
 * inr_virtual_loss -- the virtual loss of Eq. 3 together with its gradient (Eq. 2):
 *   value_out[0] = scale * sum_{k < n_idx} v[idx[k]] f(x_{idx[k]})   (FP64 device scalar,
 *   overwritten), and grad_f64 / grad_f32 exactly as inr_weighted_vjp.
 *   The value comes from the forward pass that the VJP already runs at the listed points
 *   (v is held constant, as in Eq. 3), so it costs one small reduction more than
 *   inr_weighted_vjp.  Arguments, workspace (inrct_vjp_ws_bytes), index semantics and
 *   errors as inr_weighted_vjp; value_out must not be NULL.
 */
int inr_virtual_loss(const inrct_mlp* mlp, const float* theta, const inrct_grid* grid,
                     const int32_t* idx, int64_t n_idx, const float* v, double scale,
                     double* value_out, double* grad_f64, float* grad_f32, void* ws, size_t ws_bytes,
                     cudaStream_t stream);

/*
 * grad_step -- Algorithm 1 followed by one Adam update (Sec. 4 trains with Adam):
 *   x = E{f_theta}; z = P x; r = dL/dz; v = P^T r; g = scale * sum_{i in I} v_i grad f(x_i);
 *   theta <- Adam(theta, g).
 *   theta[p] FP32 in/out; y[m] FP32; idx[n_idx] int32; adam_m, adam_s[p] FP32
 *   in/out (zero before the first step); loss_out: one FP64 device scalar
 *   (the loss at the incoming theta), may be NULL; grad_out[p] FP64 device
 *   copy of g, may be NULL.  loss selects LS or FLS.  If adam is NULL theta
 *   is not updated.  ws: at least inrct_step_ws_bytes(...) bytes.
 */
size_t inrct_step_ws_bytes(const inrct_geom* geom, const inrct_grid* grid, const inrct_mlp* mlp,
                           int64_t n_idx);
int grad_step(const inrct_geom* geom, const inrct_grid* grid, const inrct_mlp* mlp, int loss,
              float* theta, const float* y, const int32_t* idx, int64_t n_idx, double scale,
              const inrct_adam* adam, float* adam_m, float* adam_s, double* loss_out,
              double* grad_out, void* ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/*
 * Batched independent problems -- one step of Algorithm 1 plus Adam for each of
 * n_probs unrelated reconstructions (own geometry, grid, parameters, data), all
 * sharing one INR architecture.  The paper trains one problem at a time; running
 * many small ones together is this library's own addition, so that problems far
 * smaller than the GPU still fill it.
 *
 * inrct_batch_create first tunes the projector launch shapes of every geometry
 * that has no tuned plan yet (inrct_tune, using that problem's part of ws and an
 * internal stream, synchronously), then records the whole batched step once as
 * a CUDA graph with
 * one branch per problem (branches run concurrently on internal streams); each
 * grad_step_batched call launches that graph on `stream`.  Every pointer in the
 * problem table is captured: the caller keeps the buffers alive and at the same
 * addresses for the lifetime of the batch, and may change their CONTENTS
 * between launches (new index sets in idx, new data in y).
 *
 * The Adam step index lives in device memory: *step_counter (one int64, device)
 * is advanced by one at the start of every launch and read by the Adam update,
 * which therefore sees t = (previous value) + 1.  Set it to 0 before the first
 * launch.  The update is bit-identical to grad_step with adam->t equal to that t
 * (for the hash-encoded INR up to the order of its table-gradient atomics).
 *
 * Problem table entries (inrct_problem) are copied; theta, y, idx, adam_m,
 * adam_s, loss_out (nullable) have the meaning and layout of grad_step.
 * ws: at least inrct_batch_ws_bytes(...) bytes of device memory, owned by the
 * caller, kept alive with the batch.  Errors: INVALID_ARG for a bad problem
 * (its index in the message), WORKSPACE, UNSUPPORTED (an architecture the
 * selected precision cannot run), CUDA (graph capture or instantiation).
 * inrct_batch_destroy frees the graph and the internal streams (host side only).
 */
typedef struct {
  inrct_geom geom;
  inrct_grid grid;
  float* theta;
  const float* y;
  const int32_t* idx;
  int64_t n_idx;
  double scale;          /* n / |I| for the estimator of Eq. 2 */
  float* adam_m;
  float* adam_s;
  double* loss_out;      /* nullable */
} inrct_problem;

typedef struct inrct_batch inrct_batch;

size_t inrct_batch_ws_bytes(const inrct_mlp* mlp, const inrct_problem* probs, int n_probs);
int inrct_batch_create(const inrct_mlp* mlp, int loss, const inrct_problem* probs, int n_probs,
                       const inrct_adam* adam, long long* step_counter, void* ws, size_t ws_bytes,
                       inrct_batch** out);
int grad_step_batched(inrct_batch* batch, cudaStream_t stream);
int inrct_batch_destroy(inrct_batch* batch);

/* ------------------------------------------------------------------------ */
/*
 * inrct_check_index_set -- validation of an index set I, off the hot path (the
 * compute calls accept any list: out-of-range indices and points outside the
 * field of view contribute nothing, repeats count once per listing).  Writes
 * counts[0] = entries outside [0, n), counts[1] = entries outside the grid's
 * field of view (fov = 1 only), counts[2] = entries repeating an earlier one
 * (host array of 3).  idx: n_idx int32 on the device.  ws: at least
 * inrct_check_index_ws_bytes(grid) bytes of device memory (a bitmap of n bits).
 * Synchronises `stream`.
 */
size_t inrct_check_index_ws_bytes(const inrct_grid* grid);
int inrct_check_index_set(const inrct_grid* grid, const int32_t* idx, int64_t n_idx, long long* counts,
                          void* ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/*
 * Autotuning of the projector launch shapes.  The paper fixes no projector
 * implementation; this is a calling convention of this library only.
 *
 * A plan is the launch shape of project()/backproject() for one geometry: the
 * ray segments per block of the forward projector (2-D: 4, 8 or 16; cone: 2, 4
 * or 8, or 1: whole rays, 32 detector columns by 4 detector rows per block, the cone default),
 * the view splits of the 2-D adjoint (1 up to twice the default, at most
 * n_views / 8) and the voxels per thread along z of the cone adjoint (4, 8, 16 or 32; or 0,
 * one warp per (x, y) column of the volume, for N <= 512 and at most 1024 detector rows, the
 * default where it applies).
 * Every plan computes the same operator; plans differ only in the order of FP32
 * additions (results agree to rounding).
 *
 * inrct_tune times every candidate plan for (geom, grid) on `stream` (5 calls
 * each after one untimed call, on synthetic data in ws) and keeps the fastest
 * in a process-wide table keyed by the geometry kind, N, n_views, n_bins_u and
 * n_bins_v; project, project_noalloc, backproject, grad_step and the batched
 * step consult that table from then on (defaults without an entry).  The call
 * synchronises `stream` and must not run during stream capture
 * (INRCT_ERR_INVALID_ARG).  ws: at least inrct_tune_ws_bytes(geom, grid) bytes
 * of device memory, overwritten.  Workspace sizes of the other calls already
 * cover every candidate plan, so no workspace needs to grow after tuning.
 * inrct_tune_plan writes the plan in use (tuned = 1 when it came from the
 * table, 0 for the defaults); inrct_tune_set pins a plan of the caller's choice
 * (INRCT_ERR_INVALID_ARG unless every field is a candidate for the geometry);
 * inrct_tune_reset empties the table.
 */
size_t inrct_tune_ws_bytes(const inrct_geom* geom, const inrct_grid* grid);
int inrct_tune(const inrct_geom* geom, const inrct_grid* grid, void* ws, size_t ws_bytes,
               cudaStream_t stream);
int inrct_tune_plan(const inrct_geom* geom, const inrct_grid* grid, int* seg, int* bp_splits,
                    int* zc, int* tuned);
int inrct_tune_set(const inrct_geom* geom, const inrct_grid* grid, int seg, int bp_splits, int zc);
int inrct_tune_reset(void);

/* ------------------------------------------------------------------------ */
/*
 * Device-side failure reporting (not part of the method).  Every wait of the
 * tensor-core kernels (the BF16 path of inr_eval_grid, inr_weighted_vjp,
 * inr_virtual_loss, grad_step, grad_step_batched, and inrct_gemm_tn) on an mbarrier is
 * bounded: when a wait runs past the limit, the kernel records a code in a status word
 * of the device, stops its other roles, waits (bounded) for its own copies and MMAs in
 * flight, releases its tensor memory and returns, so the context stays usable; the
 * call itself has already returned INRCT_OK (launches are asynchronous).
 *
 * inrct_device_status synchronises `stream`, then reads and clears the status word of
 * the current device: INRCT_OK if no wait gave up since the last check, else
 * INRCT_ERR_TIMEOUT (inrct_last_error names the kernel role and the code: 1xx
 * weight-gradient GEMM, 2xx weight producer, 3xx MMA issuer, 4xx epilogue), and the
 * outputs of the tensor-core calls since the last check must be discarded.
 * INRCT_ERR_CUDA for code 901 (a kernel found its shared memory misaligned and did
 * nothing) or a failing CUDA call.
 *
 * inrct_set_wait_limit sets the limit of every bounded wait of later launches, in
 * nanoseconds (process-wide; 0 restores the default of one second).
 *
 * inrct_debug_stall_weight_loads is a test hook: while on (process-wide), the
 * tensor-core tile kernel issues no weight loads, so its MMA issuer's first wait runs
 * out.  With nothing in flight this is the safe way to exercise the timeout path.
 */
int inrct_device_status(cudaStream_t stream);
int inrct_set_wait_limit(unsigned long long ns);
int inrct_debug_stall_weight_loads(int on);

/* ------------------------------------------------------------------------ */
/* Instrumentation (host-side, not part of the method) */

/* Number of kernel launches this library has issued since it was loaded. */
long long inrct_launch_count(void);

/*
 * Stage profile of grad_step: while active, grad_step records a CUDA event on
 * its stream at each stage boundary.  inrct_profile_end synchronises the
 * device and writes, for stage k (0-based), the summed milliseconds over the
 * recorded steps between consecutive marks:
 *   0 weight preparation of the evaluation, 1 grid-evaluation MLP kernel,
 *   2 projection + loss, 3 backprojection (+ ramp filter), 4 VJP preparation,
 *   5 VJP MLP kernel, 6 weight-gradient GEMM and reductions, 7 Adam.
 * stage_ms: host array of n_stages (<= 8) doubles; steps_out (host, may be
 * NULL) receives the number of steps recorded (at most max_steps).
 */
int inrct_profile_begin(int max_steps);
int inrct_profile_end(double* stage_ms, int n_stages, int* steps_out);

/* ------------------------------------------------------------------------ */
/*
 * inrct_sincospi -- s[i] = sin(pi x[i]), c[i] = cos(pi x[i]) for x[i] in [-1, 1], computed
 * exactly as the Fourier features gamma(x) = [cos 2 pi B x; sin 2 pi B x] of the FFN
 * networks (Sec. 4) are inside the tensor-core VJP (the phase B x is first reduced
 * to t in [-1/2, 1/2], then to the nearest quarter turn, and the Taylor series of sin and
 * cos to degrees 9 and 10 are evaluated there: about 1e-7 absolute); exposed for
 * diagnostics.
 * (The grid evaluation, whose features only enter BF16 operands, takes the hardware
 * sine and cosine of 2 pi t instead.)  x, s, c:
 * n FP32 device values.  INVALID_ARG for NULL buffers or n <= 0.
 */
int inrct_sincospi(const float* x, float* s, float* c, int64_t n, cudaStream_t stream);

/*
 * inrct_gemm_tn -- the split-K tensor-core GEMM that forms the weight
 * gradients of the BF16 path (dW_l = sum over points of delta_l a_{l-1}^T,
 * Sec. 3, Eq. 2), exposed for diagnostics:
 *   C[m][n]      = sum_k X[k][m] Y[k][n]      n < N        (main block)
 *   C[m][N]      = sum_k X[k][m]                            (ones block, 16 columns; first used)
 *   C[m][N+16+c] = sum_k X[k][m] Y16[c][k]    c < 16       (K-major extra block)
 * X [K][M], Y [K][N] and Y16 [16][K] are row-major BF16 (Y16 may be NULL:
 * zeros); C [M][N+32] FP32 row-major, overwritten.  M a multiple of 128
 * (<= 4096), N in {0, 64, 128, 192, 256}.  Partials per split of K are summed
 * in FP64.  ws: inrct_gemm_tn_ws_bytes(K, M, N).
 */
size_t inrct_gemm_tn_ws_bytes(int64_t K, int M, int N);
int inrct_gemm_tn(const void* X, const void* Y, const void* Y16, int64_t K, int M, int N, float* C,
                  void* ws, size_t ws_bytes, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* INRCT_H */
