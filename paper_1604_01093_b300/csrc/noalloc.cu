// bf_dense_pair_noalloc: the dense normal-equation blocks of one frame pair without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need this: real-time loops
// that must not pay cudaMalloc's implicit device-wide synchronisation, processes whose memory
// manager has already reserved the GPU's memory for itself, and plugins that are handed their
// buffers by the application that embeds them.  They pass their inputs and the
// output buffer; every intermediate (the two frames' preprocessed planes, the ray tables, the
// work tables and the per-tile partial sums) lives in one file-scope device array of fixed size.
//
// The array is shared by every call on a device and keeps the last call's contents; each call
// overwrites all of it that it reads, so nothing has to start at zero.  Calls whose GPU work
// overlaps (for example on two streams without ordering) race on it.  The first call on a device
// looks up the array's device address (cudaGetSymbolAddress); make that first call before any
// stream capture.
#include <cmath>
#include <mutex>

#include "bf.h"
#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int NA_MAX_W = 160, NA_MAX_H = 120;
constexpr int NA_MAX_PX = NA_MAX_W * NA_MAX_H;
constexpr int NA_TILE_PX = 1200;
constexpr int NA_MAX_TILES = 2 * ((NA_MAX_PX + NA_TILE_PX - 1) / NA_TILE_PX);  // both directions
constexpr int NA_MAX_INTS = 64 + 3 * NA_MAX_TILES;

// byte offsets inside the scratch array (all multiples of 256)
constexpr size_t NA_OFF_A = 0;                                    // float4 [2][NA_MAX_PX]
constexpr size_t NA_OFF_B = NA_OFF_A + 2 * (size_t)NA_MAX_PX * 16;  // float4 [2][NA_MAX_PX]
constexpr size_t NA_OFF_K = NA_OFF_B + 2 * (size_t)NA_MAX_PX * 16;  // float kx[256], ky[256]
constexpr size_t NA_OFF_POSE = NA_OFF_K + 2048;                    // double [2][12]
constexpr size_t NA_OFF_M = NA_OFF_POSE + 256;                      // float [24]
constexpr size_t NA_OFF_PART = NA_OFF_M + 256;                      // double [NA_MAX_TILES][NPD]
constexpr size_t NA_OFF_OFF = NA_OFF_PART + (((size_t)NA_MAX_TILES * NPD * 8 + 255) / 256) * 256;  // float [36]
constexpr size_t NA_OFF_INT = NA_OFF_OFF + 256;                     // int [NA_MAX_INTS]
constexpr size_t NA_BYTES = NA_OFF_INT + (((size_t)NA_MAX_INTS * 4 + 255) / 256) * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// table slots inside the int region
enum {
  I_SLOT = 0,      // frame_slot[2] = {0, 1}
  I_VAR = 2,       // frame_var[2] = {-1, -1}
  I_PA = 4,        // pair_a = {0}
  I_PB = 5,        // pair_b = {1}
  I_PDP = 6,       // pair_dp[2] = {0, 1}
  I_SEG0 = 8,      // pair_seg0 = {0}
  I_SEG1 = 9,      // pair_seg1 = {0}
  I_DSRC = 10,     // dp_src[2] = {0, 1}
  I_DDST = 12,     // dp_dst[2] = {1, 0}
  I_DPAIR = 14,    // dp_pair[2] = {0, 0}
  I_DDIR = 16,     // dp_dir[2] = {0, 1}
  I_DT0 = 18,      // dp_tile0[2]
  I_DT1 = 20,      // dp_tile1[2]
  I_TILES = 64     // tile_dp, tile_px0, tile_px1 [n_tiles each]
};

struct NaPoses {
  double v[24];  // R row-major, t for frame i then frame j
};

// Writes the work tables, the ray tables kx/ky (FP64 then one rounding, as the context does) and
// the two poses into the scratch array.
__global__ void k_noalloc_setup(unsigned char *base, int W, int H, double fx, double fy, double cx, double cy,
                                NaPoses poses, int tiles_per_dir) {
  int *I = (int *)(base + NA_OFF_INT);
  float *kx = (float *)(base + NA_OFF_K), *ky = kx + 256;
  double *pose = (double *)(base + NA_OFF_POSE);
  const int tid = threadIdx.x;
  const int n_tiles = 2 * tiles_per_dir;
  if (tid == 0) {
    const int fixed[22] = {0, 1, -1, -1, 0, 1, 0, 1, 0, 0, 0, 1, 1, 0, 0, 0, 0, 1, 0, tiles_per_dir, tiles_per_dir,
                           n_tiles};
    for (int k = 0; k < 22; ++k) I[k] = fixed[k];
  }
  const int HW = W * H;
  for (int k = tid; k < n_tiles; k += blockDim.x) {
    const int dir = k / tiles_per_dir, r = k % tiles_per_dir;
    I[I_TILES + k] = dir;
    I[I_TILES + n_tiles + k] = r * NA_TILE_PX;
    I[I_TILES + 2 * n_tiles + k] = min(HW, (r + 1) * NA_TILE_PX);
  }
  for (int x = tid; x < W; x += blockDim.x) kx[x] = (float)(((double)x - cx) / fx);
  for (int y = tid; y < H; y += blockDim.x) ky[y] = (float)(((double)y - cy) / fy);
  if (tid < 24) pose[tid] = poses.v[tid];
}

std::mutex g_mu;
void *g_addr[256] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

void to_pose12(const double *m, double *p) {
  const double v[12] = {m[0], m[1], m[2], m[4], m[5], m[6], m[8], m[9], m[10], m[3], m[7], m[11]};
  for (int k = 0; k < 12; ++k) p[k] = v[k];
}

}  // namespace
}  // namespace bf

using namespace bf;

extern "C" bf_status bf_dense_pair_noalloc(int width, int height, double fx, double fy, double cx, double cy,
                                           float depth_min, float depth_max, const float *depth_i,
                                           const float *lum_i, const float *depth_j, const float *lum_j,
                                           const double *pose_i, const double *pose_j, const bf_solve_params *params,
                                           double *out, void *cuda_stream) {
  if (width < 8 || height < 8 || width > NA_MAX_W || height > NA_MAX_H) return BF_ERR_INVALID_ARG;
  if (!(fx > 0) || !(fy > 0) || !depth_i || !lum_i || !depth_j || !lum_j || !pose_i || !pose_j || !params || !out)
    return BF_ERR_INVALID_ARG;
  if (!(depth_min < depth_max) || !std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(fx) ||
      !std::isfinite(fy))
    return BF_ERR_INVALID_ARG;
  if (!(params->tau_dist > 0) || !std::isfinite(params->tau_dist) || !std::isfinite(params->tau_normal) ||
      !std::isfinite(params->w_dense) || !std::isfinite(params->w_photo) || !std::isfinite(params->w_geo))
    return BF_ERR_INVALID_ARG;
  // an error left pending by the caller would be reported by the first launch check below as ours:
  // refuse instead, and leave it for the caller to read
  if (cudaPeekAtLastError() != cudaSuccess) return BF_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char *base = nullptr;
  if (scratch_address((void **)&base) != cudaSuccess) {
    cudaGetLastError();
    return BF_ERR_CUDA;
  }
#define NA_LAUNCHED()                                          \
  do {                                                         \
    if (cudaGetLastError() != cudaSuccess) return BF_ERR_CUDA; \
  } while (0)
  const int HW = width * height;
  const int tiles_per_dir = (HW + NA_TILE_PX - 1) / NA_TILE_PX;
  const int n_tiles = 2 * tiles_per_dir;
  NaPoses poses;
  to_pose12(pose_i, poses.v);
  to_pose12(pose_j, poses.v + 12);
  k_noalloc_setup<<<1, 256, 0, st>>>(base, width, height, fx, fy, cx, cy, poses, tiles_per_dir);
  NA_LAUNCHED();

  const int *I = (const int *)(base + NA_OFF_INT);
  FrameStore fs;
  fs.storage = BF_STORE_FP32;
  fs.W = width;
  fs.H = height;
  fs.A = (const float4 *)(base + NA_OFF_A);
  fs.B = (const float4 *)(base + NA_OFF_B);
  fs.P16 = nullptr;
  fs.C16 = nullptr;
  fs.kx = (const float *)(base + NA_OFF_K);
  fs.ky = fs.kx + 256;
  float4 *A = (float4 *)(base + NA_OFF_A), *B = (float4 *)(base + NA_OFF_B);
  // planes of frame i into slot 0, of frame j into slot 1 (slot tables: frame_slot = {0, 1})
  launch_preprocess(depth_i, lum_i, 1, I + I_SLOT, fs, A, B, nullptr, nullptr, depth_min, depth_max, st);
  NA_LAUNCHED();
  launch_preprocess(depth_j, lum_j, 1, I + I_SLOT + 1, fs, A, B, nullptr, nullptr, depth_min, depth_max, st);
  NA_LAUNCHED();

  Tables t = {};
  t.n_frames = 2;
  t.n_pairs = 1;
  t.n_dp = 2;
  t.n_tiles = n_tiles;
  t.n_segs = 0;
  t.n_vars = 0;
  t.n_prob = 1;
  t.frame_slot = I + I_SLOT;
  t.frame_var = I + I_VAR;
  t.pair_a = I + I_PA;
  t.pair_b = I + I_PB;
  t.pair_dp = I + I_PDP;
  t.pair_seg0 = I + I_SEG0;
  t.pair_seg1 = I + I_SEG1;
  t.dp_src = I + I_DSRC;
  t.dp_dst = I + I_DDST;
  t.dp_pair = I + I_DPAIR;
  t.dp_dir = I + I_DDIR;
  t.dp_tile0 = I + I_DT0;
  t.dp_tile1 = I + I_DT1;
  t.tile_dp = I + I_TILES;
  t.tile_px0 = I + I_TILES + n_tiles;
  t.tile_px1 = I + I_TILES + 2 * n_tiles;
  t.seg_pair = t.seg_off = t.seg_cnt = t.seg_swap = I;
  t.n_wi = 0;
  const double *pose = (const double *)(base + NA_OFF_POSE);
  float *pairM = (float *)(base + NA_OFF_M);
  double *part = (double *)(base + NA_OFF_PART);
  launch_pair_xform(t, pose, pairM, st);
  NA_LAUNCHED();
  Intr in;
  in.fx = (float)fx;
  in.fy = (float)fy;
  in.cx = (float)cx;
  in.cy = (float)cy;
  in.W = width;
  in.H = height;
  Gates g;
  g.tau_d2 = (float)(params->tau_dist * params->tau_dist);
  g.tau_n = (float)params->tau_normal;
  launch_dense<double>(MODE_ACCUM, t, fs, in, pairM, g, (float)(params->w_dense * params->w_geo),
                       (float)(params->w_dense * params->w_photo), part, nullptr, st);
  NA_LAUNCHED();
  launch_pair_merge<double, double>(t, pose, part, nullptr, out, out + PAIRBLK, (float *)(base + NA_OFF_OFF), st);
  NA_LAUNCHED();
#undef NA_LAUNCHED
  return BF_OK;
}
