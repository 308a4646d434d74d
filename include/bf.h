/*
 * bf.h -- C ABI of the B300 global pose alignment library.
 *
 * The library implements the global pose alignment of BundleFusion (Dai et al.,
 * "BundleFusion: Real-time Globally Consistent 3D Reconstruction using
 * On-the-fly Surface Re-integration", Sec. 4.2-4.4): a Gauss-Newton solve whose
 * normal equations J^T J dX = -J^T F are solved by a preconditioned conjugate
 * gradient, over 6-DoF camera poses, minimising
 *     E_align = w_sparse E_sparse + w_dense (w_photo E_photo + w_geo E_geo)
 * in the paper's two-level form: chunk ("local") solves, then a global solve over
 * chunk keyframes.
 *
 * Conventions (Sec. 4):
 *   - A pose T_i maps camera i coordinates to world coordinates, p_w = R_i p + t_i.
 *     Poses cross the ABI as 16 doubles, a row-major 4x4 matrix [R t; 0 0 0 1].
 *   - Pixel (x, y) has its centre at integer coordinates; back-projection is
 *     ((x - cx) z / fx, (y - cy) z / fy, z) with z the depth in metres.
 *   - Images are row-major H x W float32 arrays, one per frame, frames contiguous.
 *   - The first frame of every solve is the gauge frame and stays fixed (Sec. 4.3).
 *
 * Errors: every call returns a bf_status and never throws or aborts.  On failure
 * bf_last_error() returns a message describing the most recent error of that
 * context.  A context is not thread-safe: use one context per host thread or
 * serialise the calls.  All device work of a context runs on its stream; calls
 * that return results to host memory synchronise that stream before returning.
 *
 * Ownership: host inputs are copied before the call returns and may be reused at
 * once.  Device inputs are read by work enqueued on the context's stream: they must
 * stay unchanged until that stream has executed the call's work (no extra
 * synchronisation is needed when the caller works on the same stream).  Output
 * buffers are owned by the caller.  The library owns all device memory it allocates for a context and
 * frees it in bf_destroy().
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_ctx bf_ctx;

typedef enum {
  BF_OK = 0,
  BF_ERR_INVALID_ARG = 1,   /* bad pointer, size, id or parameter                         */
  BF_ERR_OUT_OF_MEMORY = 2, /* the context's HBM budget or the device is exhausted         */
  BF_ERR_CUDA = 3,          /* a CUDA runtime call failed; see bf_last_error()             */
  BF_ERR_NOT_FOUND = 4,     /* an unknown frame id / ticket                                */
  BF_ERR_SINGULAR = 5,      /* reserved: a 6x6 block was not SPD (reported as a stats flag) */
  BF_ERR_TIMEOUT = 6,       /* a bounded wait (host or device) expired                     */
  BF_ERR_BUSY = 7           /* the request queue is full                                   */
} bf_status;

enum { BF_PTR_HOST = 0, BF_PTR_DEVICE = 1 };

/* Frame storage type of the preprocessed planes (depth, normal, I, grad I).
 *   BF_STORE_FP32: two float4 planes, 32 bytes per pixel.
 *   BF_STORE_BF16 / BF_STORE_FP16: one 16-byte record per pixel; depth stays FP32 (the dense
 *   association decisions read it), normal, I and grad I are rounded to nearest-even 16-bit
 *   values after being computed in FP32.  Halves the frame footprint and the dense term's
 *   frame traffic.  The paper keeps FP32 frames; this is a memory-layout option. */
enum { BF_STORE_FP32 = 0, BF_STORE_BF16 = 1, BF_STORE_FP16 = 2 };

/* PCG preconditioner: 6x6 block-Jacobi (default) or the paper's scalar Jacobi (Sec. 4.4). */
enum { BF_PRECOND_BLOCK_JACOBI = 0, BF_PRECOND_JACOBI = 1 };

/* Solver arithmetic.  Both evaluate residuals and Jacobians in FP32.
 *   BF_PREC_MIXED: per-tile FP32 tree sums merged in FP64; 6x6 blocks and the sums of the PCG
 *                  dot products above the warp in FP64; pose composition in FP64.  PCG vectors,
 *                  their element updates, alpha and beta (quotients of the FP64 sums) and the
 *                  block-Jacobi inverse are FP32.
 *   BF_PREC_FP32:  the plain path, FP32 throughout except the FP64 pose composition. */
enum { BF_PREC_MIXED = 0, BF_PREC_FP32 = 1 };

/* Stats flags */
enum {
  BF_FLAG_SINGULAR_BLOCK = 1, /* a diagonal 6x6 block was not SPD: scalar Jacobi used for it */
  BF_FLAG_EMPTY_FRAME = 2,    /* a frame had no constraint: marked invalid, update kept at 0 (Sec. 4.4.1) */
  BF_FLAG_PCG_BREAKDOWN = 4   /* PCG stopped early on p.Ap <= 0 */
};

typedef struct {
  int device;               /* CUDA device ordinal                                      */
  int width, height;        /* frame size (every frame of a context has this size)     */
  double fx, fy, cx, cy;    /* pinhole intrinsics of that frame size                   */
  float depth_min;          /* depth is valid iff finite and depth_min < D < depth_max */
  float depth_max;
  int storage;              /* BF_STORE_*                                              */
  size_t hbm_budget_bytes;  /* cap on the context's device allocations, 0 = no cap     */
  void *cuda_stream;        /* cudaStream_t to run on; NULL = the context creates one  */
  int max_frames_hint;      /* initial frame-store capacity (grows on demand)          */
} bf_config;

typedef struct {
  int n_gn;                 /* Gauss-Newton iterations (1..BF_MAX_GN)                  */
  int n_pcg;                /* PCG iterations per Gauss-Newton iteration (>= 0)        */
  double w_sparse, w_dense, w_photo, w_geo; /* energy weights (Sec. 4.3)               */
  int dense_ramp;           /* w_dense(k) = w_dense (k+1)/n_gn if set (Sec. 4.3: linearly increased) */
  double tau_dist;          /* dense distance gate, metres (default 0.15)              */
  double tau_normal;        /* dense normal gate, cosine (default 0.9)                 */
  double max_angle_deg;     /* dense pair set E: view directions within (default 60)   */
  int precond;              /* BF_PRECOND_*                                            */
  int dense_on;             /* evaluate the dense term (Sec. 4.3: the paper runs the global
                               dense solve only at the end of scanning)               */
  int warm_start;           /* local solves: start from the chunk's previous local poses */
  int precision;            /* BF_PREC_*                                               */
  int use_graph;            /* replay the Gauss-Newton loop as a captured CUDA graph   */
  int tile_px;              /* source pixels per dense work item; 0 = the fixed rule (target
                               frame staged in shared memory when it fits, else 4800-pixel
                               tiles); BF_TILE_AUTOTUNE = timed choice, see bf_tuned_tile_px */
  int pcg_variant;          /* BF_PCG_*: which PCG kernel runs (results agree to rounding) */
  /* Sec. 4.4.1 correspondence pruning.  prune_rmax > 0: after a solve whose r_max (largest
   * ||T_i p - T_j q|| over its sparse correspondences) exceeds prune_rmax, every
   * correspondence of the pair holding it is removed from the context and the problem is
   * solved again from the same initial poses; at most prune_rounds re-solves.  Frames left
   * without any pair are reported invalid (they keep their initial pose).  In a batch only the
   * chunks that need it are re-solved.  0 = off (the paper uses 0.05 m; 0.16 m for Kinect). */
  double prune_rmax;
  int prune_rounds;
  /* BF_SPARSE_*: how PCG applies the sparse term.  BLOCKS (default): its 6x6 pair blocks are
   * formed once per Gauss-Newton iteration and assembled with the dense ones.  MATFREE: Sec. 4.4's
   * own scheme, J p then J^T (J p) over the correspondences in every PCG iteration; the assembled
   * blocks hold the dense term alone (the preconditioner and right-hand side still include the
   * sparse term).  MATFREE runs on the grid-cooperative kernel for one problem with at least 32
   * free frames (AUTO or GRID) and on the per-problem kernel otherwise; the cluster kernel does
   * not offer it.  Both give the same step up to FP32 rounding. */
  int sparse_mode;
  /* 1: run the whole Gauss-Newton loop (all iterations, the final energy) as ONE persistent
   * kernel launch whose CTAs take tiles, segments and per-problem solves from a device work
   * queue, so independent problems (chunks, Sec. 4.2) advance at their own pace; results are
   * bitwise those of the launch sequence.  Applies to the tiled dense decomposition (tile_px > 0
   * or BF_TILE_AUTOTUNE choosing tiles, or frames too large to stage in shared memory), the
   * per-problem PCG kernel (every problem of a batch, or pcg_variant BF_PCG_CTA) and assembled
   * sparse blocks; otherwise the launch sequence runs.  A wait inside it that runs out ends
   * the solve with BF_ERR_TIMEOUT. */
  int persistent;
  /* 1: the dense term's per-thread FP32 sums are compensated (Kahan): each run of additions errs by
   * O(ulp) instead of O(n ulp), at about twice the dense kernel's instructions; always the tiled
   * dense kernel; not with persistent.  0 (default): plain FP32 runs of at most tile_px / 256
   * pixels per thread. */
  int compensated;
  /* Tensor-core dense sums (a measured alternative, not the default): 1 or 3 forms each dense
   * tile's J^T W J and J^T W r sums with tcgen05 MMAs (TF32 operands, FP32 accumulators in tensor
   * memory) instead of per-thread FP32 fused multiply-adds; 1 rounds the operands to TF32, 3
   * splits each into two TF32 parts and adds three products (close to FP32 products).  The
   * association and the residuals are unchanged.  Always the tiled dense kernel; not with
   * persistent or compensated; a solve that records its association uses the FP32 sums.  0
   * (default): off. */
  int dense_tc;
} bf_solve_params;

enum { BF_SPARSE_BLOCKS = 0, BF_SPARSE_MATFREE = 1 };

/* tile_px value asking the library to time the candidate dense work decompositions on the
 * first solve of the context (per frame size and storage) and keep the fastest. */
#define BF_TILE_AUTOTUNE (-1)

/* PCG kernels: AUTO picks CLUSTER for one large problem, else one CTA per problem. */
enum { BF_PCG_AUTO = 0, BF_PCG_CTA = 1, BF_PCG_GRID = 2, BF_PCG_CLUSTER = 3 };

#define BF_MAX_GN 64
#define BF_MAX_PRUNE 32

typedef struct {
  int n_gn_done;
  double energy[BF_MAX_GN + 1];     /* before each GN step, then after the last one     */
  double e_sparse[BF_MAX_GN + 1];   /* sum_corr w_c ||r||^2 (unweighted by w_sparse)    */
  double e_photo[BF_MAX_GN + 1];    /* sum r_photo^2                                    */
  double e_geo[BF_MAX_GN + 1];      /* sum r_geo^2                                      */
  long long n_dense_valid[BF_MAX_GN + 1]; /* associated pixels over both directions   */
  double r_max;                     /* largest ||T_i p - T_j q|| at the final poses      */
  int r_max_pair[2];                /* frame ids of the pair holding it                  */
  int n_frames, n_pairs, n_dense_pairs;
  long long n_corr;
  int flags;                        /* BF_FLAG_*                                         */
  double ms;                        /* wall time of the solve on the host (all rounds)  */
  int solves;                       /* solves run (1 + re-solves after pruning)         */
  int n_pruned;                     /* pairs removed by pruning, in order ...           */
  int pruned_pairs[2 * BF_MAX_PRUNE]; /* ... their frame ids (first BF_MAX_PRUNE pairs)  */
  int n_invalid;                    /* frames other than the first left without a pair  */
  int invalid_frames[BF_MAX_PRUNE]; /* their ids (first BF_MAX_PRUNE)                   */
} bf_solve_stats;

/* Fill defaults: 640x480 Kinect-like intrinsics scaled to 80x60, depth 0.1..10 m, FP32. */
void bf_default_config(bf_config *cfg);
/* Fill defaults: 4 GN x 10 PCG, w_sparse 1, w_dense 0.5, w_photo 0.1, w_geo 1, gates
 * 0.15 m / 0.9 / 60 deg (Sec. 4.1.1 and 4.3), block-Jacobi, dense on, mixed precision. */
void bf_default_params(bf_solve_params *p);
const char *bf_status_string(bf_status s);

/* Create a context on cfg->device.  *out receives the handle. */
bf_status bf_create(const bf_config *cfg, bf_ctx **out);
/* Destroy a context and free its device memory.  NULL is a no-op. */
bf_status bf_destroy(bf_ctx *ctx);
const char *bf_last_error(bf_ctx *ctx);

/*
 * Add (or replace) frames first_id .. first_id+n-1 (Sec. 4, input stream S = {f_i}).
 *   depth, lum: n x H x W float32 (metres; luminance), host or device per ptr_kind.
 *   init_pose:  n x 16 doubles (camera->world), host, nullable.  When given it becomes the
 *               frame's world pose (initial estimate of a global solve).
 * The frames are preprocessed on the device (Sec. 4.1.1 cached frames): validity, normals,
 * I = |grad L| and grad I, stored per the context's storage type.
 */
bf_status bf_add_frames(bf_ctx *ctx, int first_id, int n, const float *depth, const float *lum,
                        int ptr_kind, const double *init_pose);

/*
 * Append n sparse correspondences between frames frame_i != frame_j (Sec. 4.3, sparse term).
 *   p_i: n x 3 float32 points in camera i; p_j: n x 3 float32 points in camera j.
 *   weight: n float32 per-correspondence weights, nullable (= 1).
 * Host or device per ptr_kind.  Frames need not exist yet.
 */
bf_status bf_add_correspondences(bf_ctx *ctx, int frame_i, int frame_j, int n, const float *p_i,
                                 const float *p_j, const float *weight, int ptr_kind);
/*
 * Append correspondences of many pairs in one call (one host->device copy per array).
 *   pair_ids: host, 2 x n_pairs frame ids (i, j) per pair; offsets: host, n_pairs + 1 prefix
 *   counts; p_i, p_j: offsets[n_pairs] x 3 float32; weight: offsets[n_pairs] float32, nullable.
 * p_i / p_j / weight are host or device per ptr_kind.  Equivalent to one
 * bf_add_correspondences call per pair, in order.
 */
bf_status bf_add_correspondences_batch(bf_ctx *ctx, int n_pairs, const int *pair_ids, const int *offsets,
                                       const float *p_i, const float *p_j, const float *weight, int ptr_kind);
/* Drop every correspondence of the unordered pair (i, j) (Sec. 4.4.1 pruning). */
bf_status bf_remove_pair(bf_ctx *ctx, int frame_i, int frame_j);
/* Drop all correspondences of the context. */
bf_status bf_clear_correspondences(bf_ctx *ctx);

/*
 * Local (intra-chunk) solve, Sec. 4.2: frame_ids[0] is the chunk's keyframe and stays fixed;
 * the other frames start at identity (or, with warm_start, at the chunk's previous local
 * poses, Sec. 4.4).  Every correspondence pair within the chunk is used; the dense set E is
 * the pairs within max_angle_deg at the initial poses.  Local poses are stored under chunk_id.
 * A pair with fewer than 3 correspondences makes the call fail with BF_ERR_INVALID_ARG.
 * stats: nullable.
 */
bf_status bf_solve_local(bf_ctx *ctx, int chunk_id, const int *frame_ids, int n,
                         const bf_solve_params *params, bf_solve_stats *stats);

/*
 * Many independent local solves in one batched launch sequence (one problem per chunk).
 *   chunk_ids: n_chunks ids; frame_ids: concatenated frame lists; offsets: n_chunks + 1.
 *   stats: nullable, else n_chunks entries.
 */
bf_status bf_solve_local_batch(bf_ctx *ctx, int n_chunks, const int *chunk_ids, const int *frame_ids,
                               const int *offsets, const bf_solve_params *params, bf_solve_stats *stats);

/*
 * Global (inter-chunk) solve over keyframes, Sec. 4.2: keyframe_ids[0] stays fixed.  A
 * keyframe's initial pose is its world pose if it has one, else the previous keyframe's
 * pose composed with the intra-chunk delta of the chunk that links them (Sec. 4.2).
 * Afterwards every keyframe holds its optimised world pose.  stats: nullable.
 */
bf_status bf_solve_global(bf_ctx *ctx, const int *keyframe_ids, int n, const bf_solve_params *params,
                          bf_solve_stats *stats);

/*
 * World poses of frames (n x 16 doubles, host).  A chunk member's pose is its keyframe's
 * world pose composed with its local pose, T_kf T_local (Sec. 4.2); a frame outside any
 * solved chunk returns its own world pose (identity if never set).
 */
bf_status bf_get_poses(bf_ctx *ctx, const int *frame_ids, int n, double *out);

/*
 * Normal equations at given poses without solving (Sec. 4.4: J^T J dX = -J^T F), for
 * inspection and testing.  frame_ids[0] is the gauge.  poses: n x 16 host doubles.
 *   A: (6(n-1))^2 host doubles, row-major; b: 6(n-1) host doubles (= -J^T W r);
 *   energy4: host [E_total, e_sparse, e_photo, e_geo]; n_dense: host, nullable.
 * The dense term uses w_dense as given (no ramp).
 */
bf_status bf_build_system(bf_ctx *ctx, const int *frame_ids, int n, const double *poses,
                          const bf_solve_params *params, double *A, double *b, double *energy4,
                          long long *n_dense);

/*
 * Preprocessed planes of one frame, as float32 host array 7 x H x W:
 * depth (0 = invalid), normal x, y, z (0,0,0 = invalid), I, I_x, I_y.
 */
bf_status bf_get_frame_planes(bf_ctx *ctx, int frame_id, float *out);

/*
 * Dense association of frame_i's pixels into frame_j at the given poses (16 doubles each),
 * as decided by the dense kernel: out_target[k] = ny*W + nx of the nearest target pixel, or -1
 * if pixel k is rejected.  H*W int32 host output.
 */
bf_status bf_debug_association(bf_ctx *ctx, int frame_i, int frame_j, const double *pose_i,
                               const double *pose_j, const bf_solve_params *params, int32_t *out_target);

/*
 * Association recording (debug; the parity protocol of the tests, Sec. 4.3 dense matching).
 * While enabled, solves of a single problem (bf_solve_local, bf_solve_global; not batches, not
 * serving) run kernel by kernel (no graph, no persistent launch) and record, for every dense
 * evaluation e (e < n_gn: the linearisation of Gauss-Newton iteration e; e = n_gn: the final
 * energy), the associated target pixel of every source pixel of every directed pair, and the poses
 * the evaluation used.  The last such solve's record stays on the host until the next one.
 * Device memory: (n_gn + 1) x directed pairs x H x W ints while a solve runs.  Disabling frees it.
 */
bf_status bf_debug_record_association(bf_ctx *ctx, int enable);
/* The recorded association of directed pair frame_i -> frame_j (source i) at evaluation eval:
 * out_target (host, H x W int32): target pixel index y W + x, or -1; pose_i, pose_j (host, 16
 * doubles each, row-major camera -> world as the solve held them; nullable).  BF_ERR_NOT_FOUND if
 * nothing was recorded or the pair was not a dense pair of the recorded solve. */
bf_status bf_debug_recorded_association(bf_ctx *ctx, int eval, int frame_i, int frame_j, int32_t *out_target,
                                        double *pose_i, double *pose_j);

/* Debug probe of the tensor-core dense sums (no counterpart in the paper): stages given rows
 * exactly as the tcgen05 dense kernel does and returns its whole 64 x 64 FP32 accumulator as
 * held in tensor memory.  fa, fb: host arrays [8][n_rows][8] (subset, row, feature) of the A
 * (weighted) and B rows, n_rows a positive multiple of 64 up to 65536; passes 1 or 3 (as
 * bf_solve_params.dense_tc); out: host array [128][64], tensor-memory lane x column (lanes that
 * hold no accumulator row come back as the tensor memory held them).  Runs one CTA on the
 * current device with its own temporary device buffers; synchronous.  BF_ERR_INVALID_ARG for
 * bad arguments, BF_ERR_TIMEOUT if a bounded wait gave up, BF_ERR_CUDA on a CUDA error. */
bf_status bf_debug_tc_probe(int n_rows, int passes, const float *fa, const float *fb, float *out);

/*
 * Kernel accounting.  Every kernel the context launches is counted; with profiling enabled the
 * context also records a CUDA event pair around each launch on its stream and sums the device
 * time per kernel class.  bf_get_profile synchronises the stream.  The pose update and the
 * per-iteration energy record run inside the PCG kernel, so BF_K_UPDATE keeps its slot but counts
 * no launches and BF_K_ENERGY counts only a solve's final energy evaluation.  BF_K_XFORM counts
 * the pair-transform launches: one per solve when every problem is solved by the per-problem PCG
 * kernel (which refreshes its pairs' transforms itself), one more per GN iteration otherwise.
 * BF_K_BATCH counts the persistent batched-solve launches (one per solve, see `persistent`).
 */
enum {
  BF_K_PREPROCESS = 0, BF_K_XFORM, BF_K_DENSE, BF_K_SPARSE, BF_K_MERGE, BF_K_ASSEMBLE, BF_K_PCG, BF_K_UPDATE,
  BF_K_ENERGY, BF_K_PACK, BF_K_VERIFY, BF_K_KEYPOINT, BF_K_TSDF, BF_K_BATCH, BF_NPROF
};
typedef struct {
  long long launches;          /* kernels launched since the last reset (always counted)  */
  long long count[BF_NPROF];   /* timed launches per class (profiling enabled)            */
  double ms[BF_NPROF];         /* summed event-timed device milliseconds per class        */
} bf_profile;
bf_status bf_set_profiling(bf_ctx *ctx, int enable);
bf_status bf_get_profile(bf_ctx *ctx, bf_profile *out);
bf_status bf_reset_profile(bf_ctx *ctx);

/*
 * Dense normal-equation blocks of one frame pair, computed without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate at the
 * point of use (real-time loops that cannot afford cudaMalloc's implicit device-wide
 * synchronisation, hosts whose memory manager already owns the device memory, plugins that are
 * handed their buffers by the application embedding them).  No context is involved and nothing
 * is allocated: intermediates live in one fixed device array built into the library (about
 * 1.25 MB per device, held until exit).
 *   width, height: 8..160 x 8..120 (anything else returns BF_ERR_INVALID_ARG);
 *   fx, fy, cx, cy: as in bf_config (fx, fy > 0);  depth_min < depth_max: the validity range;
 *   depth_i, lum_i, depth_j, lum_j: device, H x W float32 each (raw frames);
 *   pose_i, pose_j: host, 16 doubles each (camera -> world);
 *   params: host; uses tau_dist (> 0), tau_normal, w_dense, w_photo, w_geo (finite; no ramp, no
 *           angle test); anything else about them returns BF_ERR_INVALID_ARG;
 *   out: device, 124 doubles: A_ii, A_ij, A_jj (row-major 6x6), rhs_i, rhs_j (= -J^T W r),
 *        then e_sparse (0), e_photo, e_geo, associated pixels, both directions i->j and j->i;
 *   cuda_stream: cudaStream_t (NULL = legacy default stream); the call only enqueues work.
 * Errors: argument errors return BF_ERR_INVALID_ARG before any CUDA call.  A CUDA error already
 * pending on the calling thread (for example from the caller's own failed allocation) makes the
 * call return BF_ERR_CUDA without enqueuing anything and without clearing that error.  A launch
 * that fails returns BF_ERR_CUDA at once (the launch error is consumed; work enqueued before it
 * stays queued).
 * The first call on a device looks up the array's device address: make it before any stream
 * capture.  Every call on a device shares the array and leaves its contents behind; calls whose
 * GPU work overlaps race on it, so order them on one stream.
 */
bf_status bf_dense_pair_noalloc(int width, int height, double fx, double fy, double cx, double cy, float depth_min,
                                float depth_max, const float *depth_i, const float *lum_i, const float *depth_j,
                                const float *lum_j, const double *pose_i, const double *pose_j,
                                const bf_solve_params *params, double *out, void *cuda_stream);

/*
 * Serving (continuous batching on a persistent context).  Frames and correspondences are added as
 * usual (bf_add_frames / bf_add_correspondences, which may be called while serving); requests
 * name frame ids and are queued.  n_slots worker slots, each with its own stream and solve
 * workspace, take batches from the head of the queue: consecutive local requests with identical
 * parameters (up to max_batch) form one batched solve; a global request runs alone.  Batches of
 * different slots overlap on the device.  Admission follows the context's HBM budget: a batch
 * whose workspace would not fit is halved and the rest requeued.  A request's stats.ms is its
 * latency from bf_submit to completion.  Results are also stored as by bf_solve_local /
 * bf_solve_global (bf_get_poses sees them).  Adding frames that replace existing ids, growing the
 * frame store or the correspondence pool, and clearing correspondences wait until no batch is on
 * the device.
 */
enum { BF_REQ_LOCAL = 0, BF_REQ_GLOBAL = 1 };
typedef struct {
  int kind;                 /* BF_REQ_LOCAL or BF_REQ_GLOBAL                              */
  int chunk_id;             /* local requests: chunk id the local poses are stored under   */
  const int *frame_ids;     /* host, copied by bf_submit; [0] is the fixed frame           */
  int n;
  bf_solve_params params;   /* use_graph is ignored (batches differ from one another);
                               prune_rmax must be 0 (pruning is in the synchronous calls)  */
} bf_request;
/* Start n_slots (1..8) worker slots; max_batch local requests per batch; max_queue pending.
 * Each slot runs local (chunk) batches on a high-priority stream and global solves on a
 * low-priority one, so when both are on the device the short chunk kernels are scheduled first. */
bf_status bf_serve_start(bf_ctx *ctx, int n_slots, int max_batch, int max_queue);
/* Stop the workers after their current batch; pending requests complete with BF_ERR_BUSY.
 * bf_destroy stops serving too. */
bf_status bf_serve_stop(bf_ctx *ctx);
/* Queue a request; BF_ERR_BUSY if max_queue requests are already pending. */
bf_status bf_submit(bf_ctx *ctx, const bf_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (< 0: forever, 0: poll) for a request; returns its status, or
 * BF_ERR_TIMEOUT if it has not completed (the ticket stays valid), BF_ERR_NOT_FOUND for an
 * unknown or already collected ticket.  stats: nullable. */
bf_status bf_wait(bf_ctx *ctx, uint64_t ticket, int timeout_ms, bf_solve_stats *stats);

/*
 * Key-point correspondence filter and surface-area filter (Sec. 4.1.1), batched over pairs.
 * Per pair the matches (p in camera i, q in camera j) come in order of match distance; the set
 * grows one match at a time and, while the Kabsch fit q ~ R p + t over it has a residual above
 * max_residual or a condition number sigma_1/sigma_2 above max_cond (covariance of the p points,
 * of the q points, their cross-covariance), the match with the largest residual leaves the set.
 * A pair keeps its surviving matches if at least min_matches survive and the kept p points and
 * the kept q points each span at least min_area (bounding rectangle in the plane of their two
 * principal axes).  Arithmetic in FP64, one warp per pair, at most 1024 matches per pair.
 */
typedef struct {
  double max_residual;  /* metres (default 0.02)                                        */
  double max_cond;      /* default 100                                                  */
  double min_area;      /* m^2 (default 0.032)                                          */
  int min_matches;      /* N_min (default 5)                                            */
} bf_keypoint_params;
void bf_default_keypoint_params(bf_keypoint_params *p);

/*
 *   offsets: n_pairs + 1 host ints (offsets[0] = 0); p_i, p_j: offsets[n_pairs] x 3 host floats.
 *   keep: offsets[n_pairs] host bytes (out): 1 = the match survives in a kept pair.
 *   transforms: n_pairs x 16 host doubles (out, nullable): row-major T_ij of kept pairs (else 0).
 *   status: n_pairs host ints (out, nullable): 0 kept, 1 too few matches survive, 2 area too small.
 * Synchronous; needs a context only for its device and stream.
 */
bf_status bf_filter_keypoints(bf_ctx *ctx, int n_pairs, const int *offsets, const float *p_i, const float *p_j,
                              const bf_keypoint_params *params, unsigned char *keep, double *transforms,
                              int *status);

/*
 * Dense verification of frame pairs (Sec. 4.1.1) and chunk validation (Sec. 4.2).
 * Both directions of a pair are checked: every pixel with valid depth and normal is projected
 * into the other frame, matched to the nearest pixel, and kept when
 *   ||T p - q|| < tau_dist,  (R n_src) . n_dst > tau_normal,  |C_src - C_dst| < tau_color
 * (C = the luminance given to bf_add_frames).  One CTA per pair.
 */
typedef struct {
  double tau_dist;        /* metres (default 0.15)                                      */
  double tau_normal;      /* cosine (default 0.9)                                       */
  double tau_color;       /* intensity difference (default 0.1)                         */
  double max_err;         /* pair valid iff mean re-projection error <= max_err (0.075 m) */
  double min_valid_frac;  /* ... and n_ij + n_ji >= min_valid_frac * W * H (0.02)        */
} bf_verify_params;
void bf_default_verify_params(bf_verify_params *p);

typedef struct {
  int n_ij, n_ji;         /* kept correspondences per direction                         */
  double err_ij, err_ji;  /* sums of their distances ||T p - q|| (metres)               */
  double mean_err;        /* (err_ij + err_ji) / (n_ij + n_ji), +inf if none            */
  int valid;              /* the Sec. 4.1.1 decision with the given thresholds          */
} bf_verify_result;

/*
 * Verify n frame pairs.  frame_pairs: 2n frame ids (i, j); rel: n x 16 doubles, row-major
 * T_ij mapping camera-i points into camera j (e.g. from a key-point filter's Kabsch fit);
 * T_ji is its inverse.  out: n results (host).  Synchronous.
 */
bf_status bf_verify_pairs(bf_ctx *ctx, int n, const int *frame_pairs, const double *rel,
                          const bf_verify_params *params, bf_verify_result *out);

/*
 * Chunk validation (Sec. 4.2): verify every pair of a solved chunk's frames at its local poses;
 * *valid = 0 if a pair with kept correspondences has a mean error above max_err (0.05 m).
 * worst_err / worst_pair (2 frame ids): nullable.  BF_ERR_NOT_FOUND for an unsolved chunk.
 */
bf_status bf_validate_chunk(bf_ctx *ctx, int chunk_id, double max_err, const bf_verify_params *params,
                            int *valid, double *worst_err, int *worst_pair);

/*
 * TSDF reconstruction with integration and de-integration (Sec. 5), one volume per context.
 * Voxels of 8x8x8 blocks (Sec. 5.1) found through a hash table of block coordinates keep the
 * integer sums S = sum w d_q (truncated signed distance in units of 2^-20 m), W = sum w and
 * SC = sum w c_q (intensity in units of 1/65535), w = 1 per sample; the paper's running average
 * D = (D W + w d) / (W + w) (Sec. 5.2) is S 2^-20 / W, and de-integration subtracts exactly
 * what integration added.  A frame touches the blocks containing its band samples (every valid
 * pixel's ray at depths D + k voxel/2, |k voxel/2| <= mu) and updates their voxels: projective
 * distance d = D(u) - z to the nearest pixel u of the voxel centre's projection, voxels with
 * d < -mu left alone, sdf = min(d, mu), mu = trunc_voxels * voxel_size.  Depth and intensity
 * are the frame's stored planes.  Synchronous calls.
 */
typedef struct {
  double voxel_size;   /* metres (default 0.004, the paper's default)                     */
  int trunc_voxels;    /* mu in voxels (default 5)                                        */
  int table_log2;      /* hash table of 2^table_log2 slots (default 20)                    */
  int max_blocks;      /* block pool capacity (default 65536; 6 KB per block)              */
} bf_tsdf_config;
void bf_default_tsdf_config(bf_tsdf_config *p);
/* (Re)create the context's volume, empty.  BF_ERR_OUT_OF_MEMORY beyond the HBM budget. */
bf_status bf_tsdf_init(bf_ctx *ctx, const bf_tsdf_config *cfg);
/* Integrate a frame at pose (16 doubles, camera -> world; NULL = the frame's current world
 * pose) and remember that pose as its integrated pose.  A full table or pool returns
 * BF_ERR_OUT_OF_MEMORY. */
bf_status bf_tsdf_integrate(bf_ctx *ctx, int frame_id, const double *pose);
/* Remove a frame at its integrated pose (the exact inverse of its integration). */
bf_status bf_tsdf_deintegrate(bf_ctx *ctx, int frame_id);
/*
 * Sec. 5.3 update: order the integrated frames by the distance between integrated and current
 * (optimised) world pose, ||s (e_int, t_int) - s (e_opt, t_opt)||, s = (2, 2, 2, 1, 1, 1), e the
 * Euler angles of R = Rz(g) Ry(b) Rx(a); de-integrate and re-integrate the first n_fix (the paper
 * uses 10) with a non-zero distance.  frame_ids (nullable, n_fix ints) gets them in order.
 */
bf_status bf_tsdf_reintegrate(bf_ctx *ctx, int n_fix, int *frame_ids, int *n_done);
/*
 * Copy out the allocated blocks sorted by coordinate: block_coords capacity x 3 ints (bx, by,
 * bz; voxel (ix, iy, iz) of a block has centre ((8 bx + ix + 1/2) voxel_size, ...)), sums
 * capacity x 3 x 512 ints (S, W, SC per voxel, voxel index ix + 8 iy + 64 iz).  *n = the number
 * of allocated blocks (also when it exceeds capacity; capacity 0 only counts).
 */
bf_status bf_tsdf_export(bf_ctx *ctx, long long capacity, int *block_coords, int *sums, long long *n);

/* The decomposition the autotuner chose for this context's frame size and storage: 0 = target
 * frame staged in shared memory, else the tile size in pixels.  BF_ERR_NOT_FOUND before the
 * first autotuned solve.  The choice depends on timing, so two contexts may choose differently
 * (their results then differ in the last bits); within a context it is fixed. */
bf_status bf_tuned_tile_px(bf_ctx *ctx, int *tile_px);

/*
 * Failure-detection self-test.  The library's device waits (the cooperative PCG's grid barrier,
 * the staged dense kernel's wait for its bulk copies, the persistent batched solve's wait for a
 * work-queue slot) give up after a bounded number of polls and the call that launched them
 * returns BF_ERR_TIMEOUT.  This call makes one such wait run out on purpose with `limit` polls
 * (1 .. 2^24): which = 0 polls a device word that nothing changes, which = 1 waits on an mbarrier
 * that nothing arrives on, which = 2 waits for a queue slot that nothing publishes.  *gave_up = 1
 * and BF_ERR_TIMEOUT when the wait ended as designed; the context stays usable.
 */
bf_status bf_selftest_wait_timeout(bf_ctx *ctx, int which, long long limit, int *gave_up);

/* Device bytes currently held by the context. */
size_t bf_device_bytes(bf_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* BF_H */
