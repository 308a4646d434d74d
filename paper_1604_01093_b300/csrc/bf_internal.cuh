// Internal declarations shared by the library's CUDA translation units.
//
// Data layout in HBM (one context):
//   frame store  A[slot][H*W] float4 = (D, n_x, n_y, n_z)   D = 0 marks invalid depth,
//                                                            n = 0 marks an invalid normal
//                B[slot][H*W] float4 = (I, I_x, I_y, 0)      I = |grad L| (Sec. 4.3)
//   (BF16/FP16 storage packs the same 7 channels into 16 bytes per pixel, see Frames16.)
//   correspondence pool  P[k] float4 = (p.xyz, w), Q[k] float4 = (q.xyz, 0), p in the camera
//                of the pair's smaller frame id, q in the larger one's.
//   per-solve workspace: tables (int32), poses (FP64, 12 per frame: R row-major, t),
//                per-work-item partial sums, per-pair 6x6 blocks, per-frame blocks, PCG vectors.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "bf.h"

namespace bf {

// One-time setup per device (a kernel attribute, an occupancy query).  Kernel attributes and
// occupancy belong to a device, so a context on a second device must do its own; the mutex lets
// the host threads of several contexts (and the serving workers) reach it at the same time.
// get(key, f): the value stored for (current device, key), computed by f() the first time.
struct PerDevice {
  std::mutex mu;
  std::map<std::pair<int, long long>, long long> v;
  template <typename F>
  long long get(long long key, F f) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    auto it = v.find({dev, key});
    if (it != v.end()) return it->second;
    const long long x = f();
    v[{dev, key}] = x;
    return x;
  }
  void set(long long key, long long x) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    v[{dev, key}] = x;
  }
};

// ---------------------------------------------------------------------------------------------
// Partial sums of one work item (a dense tile or a sparse segment), in the coordinates of the
// pair's target frame.  Every residual row r with weight w has a Jacobian of the form
// [a, v, c, -v] over (dw_src, dt_src, dw_tgt, dt_tgt) (Sec. 4.3 terms all share it: the
// translation parts are opposite), so J^T W J needs only six 3x3 sums and J^T W r three
// 3-vectors.
// ---------------------------------------------------------------------------------------------
constexpr int NPART = 57;
enum : int {
  P_AA = 0,   // sym 3x3  sum w a a^T   (xx xy xz yy yz zz)
  P_AV = 6,   // 3x3      sum w a v^T   (row-major)
  P_VV = 15,  // sym 3x3  sum w v v^T
  P_AC = 21,  // 3x3      sum w a c^T
  P_VC = 30,  // 3x3      sum w v c^T
  P_CC = 39,  // sym 3x3  sum w c c^T
  P_GA = 45,  // sum w r a
  P_GV = 48,  // sum w r v
  P_GC = 51,  // sum w r c
  P_E0 = 54,  // dense: sum r_geo^2        sparse: sum w_c ||r||^2
  P_E1 = 55,  // dense: sum r_photo^2      sparse: 0
  P_CNT = 56  // dense: associated pixels  sparse: correspondences
};
// Dense partial sums of one tile (target-camera coordinates).  For both dense residuals the
// source rotation Jacobian is a = v x t - c with t = t_ji the pair's translation in target
// coordinates (geometric: a = n' x (t - q); photometric: a = (y - t) x g), so every sum that
// involves a follows from the v / c sums and t; the pair merge rebuilds the NPART layout.
constexpr int NPD = 30;
enum : int {
  D_VV = 0,   // sym 3x3 sum w v v^T
  D_VC = 6,   // 3x3     sum w v c^T
  D_CC = 15,  // sym 3x3 sum w c c^T
  D_GV = 21,  // sum w r v
  D_GC = 24,  // sum w r c
  D_E0 = 27,  // sum r_geo^2
  D_E1 = 28,  // sum r_photo^2
  D_CNT = 29  // associated pixels
};
// Per-pair block record: A_aa, A_ab, A_bb (row-major 6x6), rhs_a, rhs_b (= -J^T W r).
constexpr int PAIRBLK = 120;
constexpr int PB_AA = 0, PB_AB = 36, PB_BB = 72, PB_RA = 108, PB_RB = 114;
// Per-pair energy record: e_sparse, e_photo, e_geo, n_dense.
constexpr int PAIREN = 4;

struct Intr {
  float fx, fy, cx, cy;  // FP32 roundings of the intrinsics
  int W, H;
};

// Storage of the preprocessed planes.
struct FrameStore {
  int storage;            // BF_STORE_*
  int W, H;
  const float4 *A;        // FP32: [slot][HW] (D, n)
  const float4 *B;        // FP32: [slot][HW] (I, Ix, Iy, 0)
  const uint4 *P16;       // BF16/FP16: [slot][HW] records {D (FP32 bits), nx | ny, nz | I, Ix | Iy}
  const unsigned short *C16;  // BF16/FP16: [slot][HW] intensity C (FP32 storage keeps it in B.w)
  const float *kx, *ky;   // kx[x] = fl32((x - cx)/fx), ky[y] = fl32((y - cy)/fy)
};

// 16-bit storage record of one pixel (16 bytes): word 0 the FP32 depth bits, words 1-3 the pairs
// (nx, ny), (nz, I), (Ix, Iy) as BF16 or FP16, low half first.  Rounding is to nearest, ties to
// even, from the FP32 values.
template <int KIND>
__device__ __forceinline__ unsigned short f32_to16(float v) {
  if (KIND == BF_STORE_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  return __half_as_ushort(__float2half_rn(v));
}
template <int KIND>
__device__ __forceinline__ float f16_to32(unsigned h) {
  if (KIND == BF_STORE_BF16) return __uint_as_float(h << 16);  // BF16 = the top half of an FP32
  return __half2float(__ushort_as_half((unsigned short)h));
}
template <int KIND>
__device__ __forceinline__ uint4 pack16(float4 a, float I, float Ix, float Iy) {
  uint4 r;
  r.x = __float_as_uint(a.x);
  r.y = (unsigned)f32_to16<KIND>(a.y) | ((unsigned)f32_to16<KIND>(a.z) << 16);
  r.z = (unsigned)f32_to16<KIND>(a.w) | ((unsigned)f32_to16<KIND>(I) << 16);
  r.w = (unsigned)f32_to16<KIND>(Ix) | ((unsigned)f32_to16<KIND>(Iy) << 16);
  return r;
}
// (D, nx, ny, nz) of a record
template <int KIND>
__device__ __forceinline__ float4 unpack16_dn(uint4 r) {
  return make_float4(__uint_as_float(r.x), f16_to32<KIND>(r.y & 0xffffu), f16_to32<KIND>(r.y >> 16),
                     f16_to32<KIND>(r.z & 0xffffu));
}
// (I, Ix, Iy, 0) of a record
template <int KIND>
__device__ __forceinline__ float4 unpack16_i(uint4 r) {
  return make_float4(f16_to32<KIND>(r.z >> 16), f16_to32<KIND>(r.w & 0xffffu), f16_to32<KIND>(r.w >> 16), 0.f);
}

// Flattened tables of one (batched) solve, all int32 device pointers.
struct Tables {
  int n_frames, n_pairs, n_dp, n_tiles, n_segs, n_vars, n_prob;
  const int *frame_slot;            // [n_frames]
  const int *frame_var;             // [n_frames]  var block index, -1 for a gauge frame
  const int *pair_a, *pair_b;       // [n_pairs]   solve-frame indices, a has the smaller local index
  const int *pair_dp;               // [n_pairs*2] directed pair a->b, b->a (or -1)
  const int *pair_seg0, *pair_seg1; // [n_pairs]   segment range
  const int *dp_src, *dp_dst, *dp_pair, *dp_dir;  // [n_dp]
  const int *dp_tile0, *dp_tile1;   // [n_dp]      tile range
  const int *tile_dp, *tile_px0, *tile_px1;       // [n_tiles]
  const int *seg_pair, *seg_off, *seg_cnt, *seg_swap;  // [n_segs]
  const int *inc_off, *inc;         // [n_vars+1], entries 2*pair + side (side 0: var is a)
  const int *inc_ov;                // [n_inc] var block of the pair's other frame, -1 for a gauge frame
  const int *var_frame;             // [n_vars]
  const int *prob_var0, *prob_var1, *prob_pair0, *prob_pair1;  // [n_prob]
  const int *prob_tile0, *prob_tile1, *prob_seg0, *prob_seg1;  // [n_prob] the problem's tiles / segments
  // target-staged dense work items (small frames): item w covers sw_dp[wi_off[w] .. wi_off[w+1]),
  // directed pairs that share one target frame
  int n_wi;
  const int *wi_off, *sw_dp;
};

struct Gates {
  float tau_d2;   // fl32(tau_dist^2)
  float tau_n;    // fl32(tau_normal)
};

enum { MODE_ACCUM = 0, MODE_ENERGY = 1, MODE_ASSOC = 2 };

// M = T_j^-1 T_i (source i, target j) from FP64 poses (R row-major, t), each entry summed left to
// right with explicit FP64 rounding and rounded once to FP32 (the association decisions depend on
// these exact values).  Entry e < 9 is R[e / 3][e % 3] = sum_k Rj[k][a] Ri[k][b]; entry 9 + a is
// t[a] = sum_k Rj[k][a] (t_i - t_j)[k].
__device__ __forceinline__ float pair_xform_entry(const double *Ti, const double *Tj, int e) {
  if (e < 9) {
    const int a = e / 3, b = e % 3;
    return (float)__dadd_rn(__dadd_rn(__dmul_rn(Tj[a], Ti[b]), __dmul_rn(Tj[3 + a], Ti[3 + b])),
                            __dmul_rn(Tj[6 + a], Ti[6 + b]));
  }
  const int a = e - 9;
  const double d0 = __dsub_rn(Ti[9], Tj[9]), d1 = __dsub_rn(Ti[10], Tj[10]), d2 = __dsub_rn(Ti[11], Tj[11]);
  return (float)__dadd_rn(__dadd_rn(__dmul_rn(Tj[a], d0), __dmul_rn(Tj[3 + a], d1)), __dmul_rn(Tj[6 + a], d2));
}

__device__ __forceinline__ void pair_xform32(const double *Ti, const double *Tj, float *M) {
#pragma unroll
  for (int e = 0; e < 12; ++e) M[e] = pair_xform_entry(Ti, Tj, e);
}

// Warp reduce-scatter of M per-lane values (M a power of two, 32 <= M <= 64): five exchange steps
// (lane offsets 16, 8, 4, 2, 1), each sending one half of the values still held to the partner
// lane and adding the half received, so a step costs one shuffle per value kept instead of a full
// butterfly per value.  Afterwards lane l holds the warp totals of indices (M / 32) l + j in
// acc[j], j < M / 32.  The order of the additions is fixed, so the result is deterministic.
template <int M>
__device__ __forceinline__ void warp_reduce_scatter(float (&acc)[M]) {
  static_assert(M == 32 || M == 64, "32 or 64 values");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, h = M / 2; o >= 1; o >>= 1, h >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = upper ? acc[k] : acc[k + h];
      const float keep = upper ? acc[k + h] : acc[k];
      acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// Load through L2 when CG (data written by another CTA of the same persistent launch, which the
// SM's L1 may hold an older copy of), a plain load otherwise.
template <bool CG, typename X>
__device__ __forceinline__ X ldx(const X *p) {
  if (CG) return __ldcg(p);
  return *p;
}

// Exp-map pose update R <- Exp(dw) R, t <- t + dt in FP64 (Rodrigues: Exp(dw) = I + A K + B K^2,
// K = [dw]x, K^2 = dw dw^T - th^2 I, A = sin(th) / th, B = (1 - cos(th)) / th^2).  For th <= 1/2
// (every step but a gross first one) A and B come from their Taylor series in th^2, eight terms
// each, the first omitted term below 1e-17 relative: FP64 runs at 1/64 of the FP32 rate on B300
// and the series needs 16 FMAs where sin, cos and two divisions need several times that.
// CG: the current pose is read through L2 (see ldx).
template <bool CG = false>
__device__ __forceinline__ void update_pose(double *T, const float *x) {
  const double w0 = x[0], w1 = x[1], w2 = x[2];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  double A, B;
  if (th2 <= 0.25) {
    // A = sum_k (-1)^k th^2k / (2k+1)!,  B = sum_k (-1)^k th^2k / (2k+2)!,  k = 0..7
    A = -1.0 / 1307674368000.0;
    A = fma(A, th2, 1.0 / 6227020800.0);
    A = fma(A, th2, -1.0 / 39916800.0);
    A = fma(A, th2, 1.0 / 362880.0);
    A = fma(A, th2, -1.0 / 5040.0);
    A = fma(A, th2, 1.0 / 120.0);
    A = fma(A, th2, -1.0 / 6.0);
    A = fma(A, th2, 1.0);
    B = -1.0 / 20922789888000.0;
    B = fma(B, th2, 1.0 / 87178291200.0);
    B = fma(B, th2, -1.0 / 479001600.0);
    B = fma(B, th2, 1.0 / 3628800.0);
    B = fma(B, th2, -1.0 / 40320.0);
    B = fma(B, th2, 1.0 / 720.0);
    B = fma(B, th2, -1.0 / 24.0);
    B = fma(B, th2, 0.5);
  } else {
    const double th = sqrt(th2);
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
  }
  const double w[3] = {w0, w1, w2};
  const double K[3][3] = {{0.0, -w2, w1}, {w2, 0.0, -w0}, {-w1, w0, 0.0}};
  double E[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double K2 = w[i] * w[j] - (i == j ? th2 : 0.0);
      E[i][j] = (i == j ? 1.0 : 0.0) + A * K[i][j] + B * K2;
    }
  double T0[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) T0[k] = ldx<CG>(T + k);
  double R[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[3 * i + j] = E[i][0] * T0[j] + E[i][1] * T0[3 + j] + E[i][2] * T0[6 + j];
#pragma unroll
  for (int k = 0; k < 9; ++k) T[k] = R[k];
  T[9] = T0[9] + (double)x[3];
  T[10] = T0[10] + (double)x[4];
  T[11] = T0[11] + (double)x[5];
}

// ------------------------------------------------------------------------- bounded waits
// Every wait of this library on another thread's or the copy engine's progress gives up after a
// bounded number of polls and reports an error instead of hanging the GPU.

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait_parity(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the given phase parity of an mbarrier; false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit) {
  for (long long k = 0; k < limit; ++k) {
    if (mbar_try_wait_parity(bar, parity)) return true;
    if (k > 64) __nanosleep(128);
  }
  return false;
}

// Spin until *word != old: the first `fast` polls back to back, then with a 64 ns back-off.
// Gives up (false) after `limit` polls, or as soon as *abort is set by another waiter.
__device__ __forceinline__ bool wait_change(const volatile unsigned *word, unsigned old, const volatile int *abort,
                                            long long limit, long long fast) {
  long long spins = 0;
  while (*word == old) {
    if (*abort) return false;
    if (++spins > limit) return false;
    if (spins > fast) __nanosleep(64);
  }
  return true;
}

// Spin until a work-queue slot's flag is set (published): the first 1024 polls back to back, then
// with a 256 ns back-off.  Gives up (false) after `limit` polls, or as soon as *abort is set.
__device__ __forceinline__ bool wait_published(const int *flag, const volatile int *abort, long long limit) {
  const volatile int *f = flag;
  for (long long k = 0; k < limit; ++k) {
    if (*f != 0) return true;
    if (*abort) return false;
    if (k > 1024) __nanosleep(256);
  }
  return false;
}

// Per-GN-iteration outputs the PCG kernels write besides the step: the problem's energy record
// (sum of its pairs' records, fixed order), the updated poses and (per-problem kernel only) the
// pair transforms of the updated poses for the next linearisation.
struct PcgOut {
  double *energy;  // [n_prob][PAIREN], nullable
  double *pose;    // poses updated in place with the step, nullable
  float *pairM;    // [n_pairs][2][12] transforms at the updated poses, nullable
};

// Matrix-free sparse term inside PCG (Sec. 4.4: the sparse residuals are not assembled; every
// PCG iteration evaluates J p, then J^T (J p)).  With P == nullptr the sparse 6x6 blocks are part
// of the assembled system (the default); otherwise the assembled off-diagonal and diagonal blocks
// the matvec reads hold the dense term alone and the sparse term is applied from the
// correspondence pool at the linearisation poses.
struct MatFree {
  const float4 *P, *Q;  // correspondence pool (p, w) / (q, 0); nullptr = off
  const double *pose;   // [n_frames][12] poses of the linearisation
  float w_sparse;
  float *mfy;           // [n_pairs][12] scratch: the pair's J^T W J d, frame a then frame b
};

// Arguments of the persistent batched solve (batch.cu): the solve's tables and workspace.
struct BatchArgs {
  Tables t;
  FrameStore fs;
  Intr in;
  Gates gates;
  const float4 *P, *Q;
  float w_sparse;
  float wg[BF_MAX_GN + 1], wp[BF_MAX_GN + 1];  // dense weights of each GN iteration; [n_gn]: final energy
  int n_gn, n_pcg, precond;
  double *pose;
  float *pairM;
  void *dpart, *spart;
  float *srmax;
  int *srarg;
  void *pairblk, *pairen;
  float *pairoff;
  void *Dd, *rhs;
  float *Df, *Minv;
  int *vflags, *pflags;
  float *x, *r, *z, *p, *q;
  double *energy;
};
// Work queue of the persistent batched solve (device memory of batch_queue_bytes()).
struct BatchQueue {
  int *head, *tail, *err;  // claim and publication counters; err: 1 a wait ran out, 2 queue overflow
  int *done;               // [n_prob] completed tiles / segments of each problem's current stage
  int *flags;              // [total] 1 once the slot's item is published
  int4 *items;             // [total] {type, problem, GN iteration, tile / segment}
  int n_prob, total;
  long long wait_limit;
};
// Items a persistent solve of problems with L_p tiles + segments publishes: per problem one
// transform item, n_gn x (L_p + 1) for the iterations, L_p + 1 for the final energy.
inline long long batch_total_items(const int *L, int n_prob, int n_gn) {
  long long total = 0;
  for (int p = 0; p < n_prob; ++p) total += 1 + (long long)n_gn * (L[p] + 1) + L[p] + 1;
  return total;
}
inline size_t batch_zero_bytes(int n_prob, long long total) {
  return ((256 + 4 * (size_t)n_prob + 4 * (size_t)total) + 255) & ~(size_t)255;
}
inline size_t batch_queue_bytes(int n_prob, long long total) {
  return batch_zero_bytes(n_prob, total) + 16 * (size_t)total;
}
// One cooperative launch (after resetting the queue's counters and flags); -1 if refused.  The
// error word (offset 8 of qmem) is nonzero after the launch if a wait gave up.
template <typename Acc>
int launch_batch(const BatchArgs &a, void *qmem, long long total, cudaStream_t st);

// ------------------------------------------------------------------ launch wrappers (host side)
// Dense verification (Sec. 4.1.1): one CTA per frame pair, both directions.  rec[p]: slots of
// the two frames, then fl32(T_ij) and fl32(T_ji) (R row-major, t); out[p] = {n_ij, n_ji, e_ij, e_ji}.
struct VerifyPair {
  int slot_i, slot_j;
  float M[2][12];
};
int launch_verify(int n_pairs, const VerifyPair *rec, const FrameStore &fs, const Intr &in, float tau_d2,
                  float tau_n, float tau_c, double *out, cudaStream_t st);
// Key-point filter (Sec. 4.1.1), one warp per pair; res: keypoint_result_bytes() per pair
// {R (9 doubles), t (3 doubles), status, pad}.  Pairs must have at most keypoint_nmax() matches.
int keypoint_nmax();
size_t keypoint_result_bytes();
int launch_keypoints(int n_pairs, const int *off, const float *P, const float *Q, double max_res, double max_cond,
                     int min_matches, double min_area, unsigned char *keep, void *res, cudaStream_t st);
// Bounded-wait self-test: which = 0 polls *word (which stays 0), 1 waits on an mbarrier nothing
// arrives on, 2 waits for a work-queue slot nothing publishes (*word as its flag); *err = 1 when
// the wait gave up after `limit` polls.
int launch_selftest_wait(int which, const unsigned *word, int *err, long long limit, cudaStream_t st);
// TSDF volume on the device (Sec. 5): hash table of packed block coordinates, block pool of
// integer sums, the touched list of the current call, counters and the error bits
// (1 probe limit, 2 pool full, 4 touched list full, 8 block coordinate out of range).
struct TsdfDev {
  unsigned long long *keys;  // [mask + 1], ~0 = empty
  int *vals;                 // [mask + 1], pool record (bit 30: fresh), -1 = none
  int *stamp;                // [mask + 1], id of the last call that touched the slot
  int *touched;              // [max_blocks] slots touched by the current call
  int *n_touched, *n_blocks, *err;
  int *S, *W, *SC;           // [max_blocks][512]
  unsigned mask;
  int max_blocks, K;
  float h, mu, inv_block, vs, inv_q;
};
struct TsdfPose {
  float R[9], t[3];  // camera -> world, rounded to FP32
};
int launch_tsdf(const TsdfDev &v, const FrameStore &fs, const Intr &in, int slot, const TsdfPose &P, int sign,
                int call_id, cudaStream_t st);
int launch_preprocess(const float *depth, const float *lum, int n, const int *slots_dev, FrameStore fs,
                       float4 *A, float4 *B, uint4 *P16, unsigned short *C16, float dmin, float dmax,
                       cudaStream_t st);
int launch_pack_corr(const float *p_i, const float *p_j, const float *w, int n, int swap, float4 *P, float4 *Q,
                      cudaStream_t st);
int launch_pair_xform(const Tables &t, const double *pose, float *pairM, cudaStream_t st);
int launch_pack_corr_batch(const float *p_i, const float *p_j, const float *w, int n_total, const int *off,
                           const int *swap, int n_pairs, float4 *P, float4 *Q, cudaStream_t st);
// Target-staged dense kernel (whole target frame in shared memory, loaded by TMA bulk copies).
// Usable when dense_staged_fits(W, H); writes one partial per directed pair.  err: device int
// set to 1 if a bulk copy did not complete within the wait limit.
bool dense_staged_fits(int W, int H, int storage);
int dense_staged_smem(int W, int H, int storage);
template <typename Part>
int launch_dense_staged(int mode, const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g,
                        float w_geo, float w_photo, Part *part, int *err, int *rec, cudaStream_t st);
template <typename Part>
int launch_dense(int mode, const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g,
                  float w_geo, float w_photo, Part *part, int *assoc, cudaStream_t st, bool comp = false);
// Tensor-core form of the dense ACCUM launch over the tiled decomposition (passes 1 or 3); sets
// *err if one of its bounded waits gave up.
template <typename Part>
int launch_dense_tc(const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g, float w_geo,
                    float w_photo, Part *part, int *err, int passes, cudaStream_t st);
template <typename Part>
int launch_sparse(int mode, const Tables &t, const float4 *P, const float4 *Q, const float *pairM, float w_sparse,
                   Part *part, float *seg_rmax, int *seg_rarg, cudaStream_t st);
template <typename Acc, typename Part>
int launch_pair_merge(const Tables &t, const double *pose, const Part *dpart, const Part *spart, Acc *pairblk,
                       Acc *pairen, float *pairoff, cudaStream_t st);
template <typename Acc>
int launch_pair_energy(const Tables &t, const Acc *dpart, const Acc *spart, Acc *pairen, cudaStream_t st);
template <typename Acc>
int launch_assemble(const Tables &t, const Acc *pairblk, int precond, Acc *Dd, Acc *rhs, float *Df, float *Minv,
                     int *vflags, cudaStream_t st);
template <typename Acc>
int launch_pcg(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs, float *x,
                float *r, float *z, float *p, float *q, int n_pcg, int *pflags, const Acc *pairen, PcgOut po,
                const MatFree &mf, cudaStream_t st);
// One large problem over many CTAs (cooperative launch).  coop_mem: coop_mem_bytes(grid) bytes
// of device memory (barrier state + per-CTA partials); its first 16 bytes are reset here.
// Returns -1 if the cooperative launch was refused.
template <typename Acc>
int launch_pcg_coop(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs,
                    float *x, float *r, float *z, float *p0, float *p1, float *q, int n_pcg, int *pflags,
                    void *coop_mem, int grid, const Acc *pairen, PcgOut po, const MatFree &mf, cudaStream_t st);
int coop_grid_size(int n_vars);
// One large problem on one thread-block cluster of cl CTAs (vectors replicated in shared memory).
// Returns -1 if the launch was refused.
template <typename Acc>
int launch_pcg_cluster(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs,
                       float *x, int n_pcg, int *pflags, int cl, const int *inc_off_host, const Acc *pairen, PcgOut po,
                       cudaStream_t st);
size_t cluster_smem_bytes(int n_vars, int cl);
// Whether the cluster PCG's CTAs can keep their incidence blocks in shared memory (inc_off: the
// host copy of the incidence offsets).
bool cluster_cache_fits(int n_vars, int cl, const int *inc_off);
int cluster_size_max();
size_t coop_mem_bytes(int grid);
template <typename Acc>
int launch_energy_reduce(const Tables &t, const Acc *pairen, double *out, cudaStream_t st);

}  // namespace bf
