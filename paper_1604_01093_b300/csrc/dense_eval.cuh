// Dense photometric + geometric term evaluation shared by the dense kernels of dense.cu and the
// persistent batched solve of solve.cu (per-pixel association, residuals, Jacobians and the
// per-tile reduction; the design notes are at the top of dense.cu).
#pragma once
#include <type_traits>

#include "bf_internal.cuh"

namespace bf {


#define FM __fmul_rn
#define FA __fadd_rn
#define FS __fsub_rn
#define FMA __fmaf_rn

struct V3 {
  float x, y, z;
};

// A stored normal (y, z, w of the record) is valid unless all three components are +-0.
__device__ __forceinline__ bool normal_valid(const float4 &a) {
  return ((__float_as_uint(a.y) | __float_as_uint(a.z) | __float_as_uint(a.w)) << 1) != 0u;
}
__device__ __forceinline__ V3 cross3(V3 a, V3 b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Per-thread dense sums.  With u = (v, c) the six Jacobian components of a row, the 21 upper-
// triangle products w u_i u_j (the VV, VC and CC sums) are kept in register pairs so that one
// packed FP32 fused multiply-add (__ffma2_rn: per component exactly __fmaf_rn) updates two of
// them: pair (i, j) with (i + 1, j + 1) for rows 0-1, 2-3 and 4-5, and the three left over
// ((0,5), (2,5), (4,5)) alone.  Every sum sees the same operations in the same order as with one
// scalar accumulator each: w u_i first, then fma(w u_i, u_j, sum).
struct DAcc {
  float2 p[9];  // (0,0)(1,1) (0,1)(1,2) (0,2)(1,3) (0,3)(1,4) (0,4)(1,5) (2,2)(3,3) (2,3)(3,4) (2,4)(3,5) (4,4)(5,5)
  float s05, s25, s45;
  float2 g[3];  // r w u: (0,1) (2,3) (4,5)
  float e0, e1, cnt;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = make_float2(0.f, 0.f);
    s05 = s25 = s45 = e0 = e1 = cnt = 0.f;
  }
  // the NPD layout (D_VV, D_VC, D_CC, D_GV, D_GC, D_E0, D_E1, D_CNT)
  __device__ __forceinline__ void to_array(float (&a)[NPD]) const {
    a[D_VV + 0] = p[0].x; a[D_VV + 1] = p[1].x; a[D_VV + 2] = p[2].x;
    a[D_VV + 3] = p[0].y; a[D_VV + 4] = p[1].y; a[D_VV + 5] = p[5].x;
    a[D_VC + 0] = p[3].x; a[D_VC + 1] = p[4].x; a[D_VC + 2] = s05;
    a[D_VC + 3] = p[2].y; a[D_VC + 4] = p[3].y; a[D_VC + 5] = p[4].y;
    a[D_VC + 6] = p[6].x; a[D_VC + 7] = p[7].x; a[D_VC + 8] = s25;
    a[D_CC + 0] = p[5].y; a[D_CC + 1] = p[6].y; a[D_CC + 2] = p[7].y;
    a[D_CC + 3] = p[8].x; a[D_CC + 4] = s45; a[D_CC + 5] = p[8].y;
    a[D_GV + 0] = g[0].x; a[D_GV + 1] = g[0].y; a[D_GV + 2] = g[1].x;
    a[D_GC + 0] = g[1].y; a[D_GC + 1] = g[2].x; a[D_GC + 2] = g[2].y;
    a[D_E0] = e0;
    a[D_E1] = e1;
    a[D_CNT] = cnt;
  }
  __device__ __forceinline__ void add_energy(float r_g, float r_p) {
    e0 = __fmaf_rn(r_g, r_g, e0);
    e1 = __fmaf_rn(r_p, r_p, e1);
    cnt += 1.f;
  }
  __device__ __forceinline__ void add_row(float w, float r, V3 v, V3 c);
};

// Accumulate one dense residual row (weight w, residual r, Jacobian [v x t - c, v, c, -v]).
__device__ __forceinline__ void accum_vc(DAcc &A, float w, float r, V3 v, V3 c) {
  const float2 U01 = make_float2(v.x, v.y), U12 = make_float2(v.y, v.z), U23 = make_float2(v.z, c.x);
  const float2 U34 = make_float2(c.x, c.y), U45 = make_float2(c.y, c.z);
  const float2 W2 = make_float2(w, w);
  const float2 WU01 = __fmul2_rn(W2, U01), WU23 = __fmul2_rn(W2, U23), WU45 = __fmul2_rn(W2, U45);
  A.p[0] = __ffma2_rn(WU01, U01, A.p[0]);
  A.p[1] = __ffma2_rn(WU01, U12, A.p[1]);
  A.p[2] = __ffma2_rn(WU01, U23, A.p[2]);
  A.p[3] = __ffma2_rn(WU01, U34, A.p[3]);
  A.p[4] = __ffma2_rn(WU01, U45, A.p[4]);
  A.p[5] = __ffma2_rn(WU23, U23, A.p[5]);
  A.p[6] = __ffma2_rn(WU23, U34, A.p[6]);
  A.p[7] = __ffma2_rn(WU23, U45, A.p[7]);
  A.p[8] = __ffma2_rn(WU45, U45, A.p[8]);
  A.s05 = __fmaf_rn(WU01.x, c.z, A.s05);
  A.s25 = __fmaf_rn(WU23.x, c.z, A.s25);
  A.s45 = __fmaf_rn(WU45.x, c.z, A.s45);
  const float2 R2 = make_float2(r, r);
  A.g[0] = __ffma2_rn(R2, WU01, A.g[0]);
  A.g[1] = __ffma2_rn(R2, WU23, A.g[1]);
  A.g[2] = __ffma2_rn(R2, WU45, A.g[2]);
}
__device__ __forceinline__ void DAcc::add_row(float w, float r, V3 v, V3 c) { accum_vc(*this, w, r, v, c); }

// The same sums with compensated (Kahan) FP32 addition: every sum carries the rounding error of
// its additions in a second register and subtracts it from the next term, so a run of n additions
// errs by O(ulp) instead of O(n ulp).  Each term (w u_i u_j, r w u_i, r^2, 1) is formed by one
// rounded multiplication and added with four rounded additions; about 2.3x the instructions and
// twice the registers of DAcc (an accuracy option, bf_solve_params.compensated).
struct DAccK {
  float s[NPD], c[NPD];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < NPD; ++k) s[k] = c[k] = 0.f;
  }
  __device__ __forceinline__ void add(int k, float t) {
    const float y = __fsub_rn(t, c[k]);
    const float n = __fadd_rn(s[k], y);
    c[k] = __fsub_rn(__fsub_rn(n, s[k]), y);
    s[k] = n;
  }
  __device__ __forceinline__ void to_array(float (&a)[NPD]) const {
#pragma unroll
    for (int k = 0; k < NPD; ++k) a[k] = s[k];
  }
  __device__ __forceinline__ void add_energy(float r_g, float r_p) {
    add(D_E0, __fmul_rn(r_g, r_g));
    add(D_E1, __fmul_rn(r_p, r_p));
    add(D_CNT, 1.f);
  }
  // u = (v, c): VV, VC, CC and the gradients in the NPD layout of DAcc::to_array
  __device__ __forceinline__ void add_row(float w, float r, V3 v, V3 cc) {
    const float u[6] = {v.x, v.y, v.z, cc.x, cc.y, cc.z};
    float wu[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) wu[i] = __fmul_rn(w, u[i]);
    int vv = D_VV, vc = D_VC, ccx = D_CC;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) add(vv++, __fmul_rn(wu[i], u[j]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 3; j < 6; ++j) add(vc++, __fmul_rn(wu[i], u[j]));
#pragma unroll
    for (int i = 3; i < 6; ++i)
#pragma unroll
      for (int j = i; j < 6; ++j) add(ccx++, __fmul_rn(wu[i], u[j]));
#pragma unroll
    for (int i = 0; i < 3; ++i) add(D_GV + i, __fmul_rn(r, wu[i]));
#pragma unroll
    for (int i = 0; i < 3; ++i) add(D_GC + i, __fmul_rn(r, wu[3 + i]));
  }
};

// Fixed-order CTA reduction of N values; thread k < N writes out[k].
// Fixed-order CTA reduction of N <= 32 values; thread k < N writes out[k].  red: shared memory
// of BS / 32 rows of N floats.  Per warp a reduce-scatter (lane l ends with value l), then the
// warps' totals in warp order.
template <int BS, int N, typename Part>
__device__ __forceinline__ void cta_reduce_store(float (&acc)[N], Part *__restrict__ out, float (*red)[N]) {
  static_assert(N <= 32, "at most 32 values");
  constexpr int NW = BS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = k < N ? acc[k] : 0.f;
  warp_reduce_scatter<32>(v);
  if (lane < N) red[warp][lane] = v[0];
  __syncthreads();
  if (threadIdx.x < N) {
    Part s = (Part)red[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < NW; ++w) s += (Part)red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Relative pose of a directed pair (FP32): y = R d + t maps source-camera to target-camera points.
struct PairXf {
  float R00, R01, R02, R10, R11, R12, R20, R21, R22, t0, t1, t2;
};

// CG: read through L2 (the transforms were written by another CTA of a persistent launch).
template <bool CG = false>
__device__ __forceinline__ PairXf load_xf(const float *M) {
  if (CG)
    return PairXf{__ldcg(M), __ldcg(M + 1), __ldcg(M + 2), __ldcg(M + 3), __ldcg(M + 4),  __ldcg(M + 5),
                  __ldcg(M + 6), __ldcg(M + 7), __ldcg(M + 8), __ldcg(M + 9), __ldcg(M + 10), __ldcg(M + 11)};
  return PairXf{M[0], M[1], M[2], M[3], M[4], M[5], M[6], M[7], M[8], M[9], M[10], M[11]};
}

// The association of a source pixel up to the target addresses (the first half of eval_pixel):
// y = R d + t, its projection u, the nearest target pixel (tx, ty) and the rotated source normal
// m.  False where the pixel has no association without reading the target (invalid source, y
// behind the camera, nearest pixel off the 3-pixel interior).
struct PixA {
  float Y0, Y1, Y2, iz, ux, uy, m0, m1, m2;
  int tx, ty;
};

__device__ __forceinline__ bool assoc_front(const float4 a, int x, int y, const PairXf &X, const Intr &in,
                                            const float *kx, const float *ky, PixA &s) {
  if (!(a.x > 0.f && normal_valid(a))) return false;
  const int W = in.W, H = in.H;
  const float z = a.x;
  // ---- association decisions, explicitly rounded FP32 in a fixed order: products, sums and
  // fused multiply-adds (one rounding of a*b + c), y = R d + t accumulated from t ----
  const float dx = FM(kx[x], z), dy = FM(ky[y], z), dz = z;
  s.Y0 = FMA(X.R02, dz, FMA(X.R01, dy, FMA(X.R00, dx, X.t0)));
  s.Y1 = FMA(X.R12, dz, FMA(X.R11, dy, FMA(X.R10, dx, X.t1)));
  s.Y2 = FMA(X.R22, dz, FMA(X.R21, dy, FMA(X.R20, dx, X.t2)));
  if (!(s.Y2 > 0.f)) return false;
  // the hardware reciprocal (rcp.approx: one MUFU instruction, about 1 ulp): the correctly rounded
  // __frcp_rn added a refinement and a slow-path test to every pixel.  Its ulp moves u by ~1e-5 px,
  // inside the FP32 tie windows of the decisions
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s.iz) : "f"(s.Y2));
  s.ux = FMA(in.fx, FM(s.Y0, s.iz), in.cx);
  s.uy = FMA(in.fy, FM(s.Y1, s.iz), in.cy);
  // nearest pixel floor(u + 0.5) on the 3-pixel interior, 3 <= n <= W - 4 (inside the image without a
  // test of its own).  Then the bilinear taps floor(u), floor(u) + 1 lie on the 2-pixel interior where
  // grad I is defined (floor(u) >= n - 1 and floor(u) + 1 <= n + 1), and every threshold on u sits at
  // a half-integer, which an integer projection (every pixel of an identity relative pose) never hits
  const float nxf = floorf(FA(s.ux, 0.5f)), nyf = floorf(FA(s.uy, 0.5f));
  if (!(nxf >= 3.f && nxf <= (float)(W - 4) && nyf >= 3.f && nyf <= (float)(H - 4))) return false;
  s.tx = (int)nxf;
  s.ty = (int)nyf;
  s.m0 = FMA(X.R02, a.w, FMA(X.R01, a.z, FM(X.R00, a.y)));
  s.m1 = FMA(X.R12, a.w, FMA(X.R11, a.z, FM(X.R10, a.y)));
  s.m2 = FMA(X.R22, a.w, FMA(X.R21, a.z, FM(X.R20, a.y)));
  return true;
}

// Bilinear base tap floor(u) as a pixel index.
__device__ __forceinline__ int assoc_tap0(const PixA &s, int W) {
  return (int)floorf(s.uy) * W + (int)floorf(s.ux);
}

// The second half: the gates on the nearest target record b = (D, n), then (MODE_ACCUM) the
// residual rows' contributions to acc.  c00..c11 = the bilinear taps' (I, Ix, Iy); srcI() gives
// the source pixel's I.  Returns the associated target pixel or -1.
template <int MODE, typename LI, typename AccT>
__device__ __forceinline__ int assoc_back(const PixA &s, const float4 b, const float4 c00, const float4 c01,
                                          const float4 c10, const float4 c11, const Intr &in, const float *kx,
                                          const float *ky, const Gates &g, LI srcI, float w_geo, float w_photo,
                                          AccT &acc) {
  if (!(b.x > 0.f && normal_valid(b))) return -1;
  const float qx = FM(kx[s.tx], b.x), qy = FM(ky[s.ty], b.x), qz = b.x;
  const float ex = FS(s.Y0, qx), ey = FS(s.Y1, qy), ez = FS(s.Y2, qz);
  const float dist2 = FMA(ez, ez, FMA(ey, ey, FM(ex, ex)));
  const float ndot = FMA(s.m2, b.w, FMA(s.m1, b.z, FM(s.m0, b.y)));
  if (!(dist2 < g.tau_d2 && ndot > g.tau_n)) return -1;
  const int tpx = s.ty * in.W + s.tx;
  if (MODE == MODE_ASSOC) return tpx;
  // ---- residuals and Jacobians (free FP32) in camera-j coordinates ----
  const float m0 = s.m0, m1 = s.m1, m2 = s.m2, Y0 = s.Y0, Y1 = s.Y1, Y2 = s.Y2, iz = s.iz;
  const float r_g = m0 * ex + m1 * ey + m2 * ez;
  const float bxf = floorf(s.ux), byf = floorf(s.uy);
  const float wx = s.ux - bxf, wy = s.uy - byf;
  const float w00 = (1.f - wx) * (1.f - wy), w01 = wx * (1.f - wy);
  const float w10 = (1.f - wx) * wy, w11 = wx * wy;
  const float Ij = w00 * c00.x + w01 * c01.x + w10 * c10.x + w11 * c11.x;
  const float gxI = w00 * c00.y + w01 * c01.y + w10 * c10.y + w11 * c11.y;
  const float gyI = w00 * c00.z + w01 * c01.z + w10 * c10.z + w11 * c11.z;
  const float r_p = srcI() - Ij;
  acc.add_energy(r_g, r_p);
  if (MODE == MODE_ACCUM) {
    // geometric: v = m, c = m x q
    const V3 m{m0, m1, m2}, q{qx, qy, qz};
    acc.add_row(w_geo, r_g, m, cross3(m, q));
    // photometric: v = g = d r_p / d y = -grad I^T Jpi(y), c = g x y
    const float gfx = gxI * in.fx * iz, gfy = gyI * in.fy * iz;
    const V3 gv{-gfx, -gfy, (gfx * Y0 + gfy * Y1) * iz};
    acc.add_row(w_photo, r_p, gv, cross3(gv, V3{Y0, Y1, Y2}));
  }
  return tpx;
}

// Evaluate source pixel (x, y) of a directed pair: association, gates and (MODE_ACCUM) the
// residual rows' contributions to acc.  a = source (D, n); loadA / loadB read the target's
// (D, n) and (I, Ix, Iy); srcI() gives the source pixel's I.  Returns the associated target
// pixel or -1.
template <int MODE, typename LA, typename LB, typename LI, typename AccT>
__device__ __forceinline__ int eval_pixel(const float4 a, int x, int y, const PairXf &X, const Intr &in,
                                          const float *kx, const float *ky, const Gates &g, LA loadA, LB loadB,
                                          LI srcI, float w_geo, float w_photo, AccT &acc) {
  PixA s;
  if (!assoc_front(a, x, y, X, in, kx, ky, s)) return -1;
  const int W = in.W;
  const int b0 = assoc_tap0(s, W);
  // issue the target reads together: nearest (D, n) and the four (I, Ix, Iy) taps
  const float4 b = loadA(s.ty * W + s.tx);
  float4 c00, c01, c10, c11;
  if (MODE != MODE_ASSOC) {
    c00 = loadB(b0);
    c01 = loadB(b0 + 1);
    c10 = loadB(b0 + W);
    c11 = loadB(b0 + W + 1);
  }
  return assoc_back<MODE>(s, b, c00, c01, c10, c11, in, kx, ky, g, srcI, w_geo, w_photo, acc);
}

// Pixel walk of one thread: px = start, start + stride, ... with (x, y) advanced incrementally.
struct PixWalk {
  int px, x, y, sx, sy, W;
  __device__ __forceinline__ PixWalk(int start, int stride, int W_) : px(start), W(W_) {
    y = start / W_;
    x = start - y * W_;
    sy = stride / W_;
    sx = stride - sy * W_;
  }
  __device__ __forceinline__ void next(int stride) {
    px += stride;
    x += sx;
    y += sy;
    if (x >= W) {
      x -= W;
      ++y;
    }
  }
};

constexpr int DENSE_BS = 256;

// One dense tile (work item = consecutive source pixels of one directed pair), evaluated by a
// CTA of DENSE_BS threads.  ktab: shared memory for kx[W] then ky[H]; red: the reduction's shared
// memory.  Ends with the CTA's partial record written by threads < NPD.
// REC (debug): also write every source pixel's associated target pixel (or -1) to
// assoc[d * H * W + px], d the tile's directed pair; MODE_ASSOC always does.  COMP: compensated
// per-thread sums (DAccK) instead of DAcc.
template <int MODE, int KIND, typename Part, bool CG = false, bool REC = false, bool COMP = false>
__device__ __forceinline__ void dense_tile(int tile, const Tables &t, const FrameStore &fs, const Intr &in,
                                           const float *__restrict__ pairM, const Gates &g, float w_geo,
                                           float w_photo, Part *__restrict__ part, int *__restrict__ assoc,
                                           float *ktab, float (*red)[NPD]) {
  const int d = t.tile_dp[tile];
  const int px0 = t.tile_px0[tile], px1 = t.tile_px1[tile];
  const int W = in.W, H = in.H;
  const long long HW = (long long)W * H;
  const int ss = t.frame_slot[t.dp_src[d]], ts = t.frame_slot[t.dp_dst[d]];
  const PairXf X = load_xf<CG>(pairM + (t.dp_pair[d] * 2 + t.dp_dir[d]) * 12);
  // the ray tables, loaded here (after X: that order keeps the register allocation of the pixel loop)
  float *kx = ktab, *ky = ktab + W;
  for (int k = threadIdx.x; k < W + H; k += DENSE_BS) ktab[k] = k < W ? fs.kx[k] : fs.ky[k - W];
  __syncthreads();
  typename std::conditional<COMP, DAccK, DAcc>::type acc;
  acc.zero();
  if (KIND == BF_STORE_FP32) {
    const float4 *__restrict__ As = fs.A + (long long)ss * HW;
    const float4 *__restrict__ Bs = fs.B + (long long)ss * HW;
    const float4 *__restrict__ At = fs.A + (long long)ts * HW;
    const float4 *__restrict__ Bt = fs.B + (long long)ts * HW;
    auto loadA = [&](int i) { return At[i]; };
    auto loadB = [&](int i) { return Bt[i]; };
    float4 a_next = make_float4(0.f, 0.f, 0.f, 0.f);
    if (px0 + (int)threadIdx.x < px1) a_next = As[px0 + threadIdx.x];
    for (PixWalk w(px0 + threadIdx.x, DENSE_BS, W); w.px < px1; w.next(DENSE_BS)) {
      const float4 a = a_next;  // prefetched one iteration ahead
      if (w.px + DENSE_BS < px1) a_next = As[w.px + DENSE_BS];
      const int px = w.px;
      auto srcI = [&]() { return Bs[px].x; };
      const int tgt = eval_pixel<MODE>(a, w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo, w_photo, acc);
      if (MODE == MODE_ASSOC || REC) assoc[(long long)d * HW + w.px] = tgt;
    }
  } else {
    const uint4 *__restrict__ Ps = fs.P16 + (long long)ss * HW;
    const uint4 *__restrict__ Pt = fs.P16 + (long long)ts * HW;
    auto loadA = [&](int i) { return unpack16_dn<KIND>(Pt[i]); };
    auto loadB = [&](int i) { return unpack16_i<KIND>(Pt[i]); };
    uint4 r_next = make_uint4(0u, 0u, 0u, 0u);
    if (px0 + (int)threadIdx.x < px1) r_next = Ps[px0 + threadIdx.x];
    for (PixWalk w(px0 + threadIdx.x, DENSE_BS, W); w.px < px1; w.next(DENSE_BS)) {
      const uint4 r = r_next;
      if (w.px + DENSE_BS < px1) r_next = Ps[w.px + DENSE_BS];
      auto srcI = [&]() { return unpack16_i<KIND>(r).x; };
      const int tgt = eval_pixel<MODE>(unpack16_dn<KIND>(r), w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo,
                                       w_photo, acc);
      if (MODE == MODE_ASSOC || REC) assoc[(long long)d * HW + w.px] = tgt;
    }
  }
  if (MODE != MODE_ASSOC) {
    float sums[NPD];
    acc.to_array(sums);
    cta_reduce_store<DENSE_BS, NPD, Part>(sums, part + (long long)tile * NPD, red);
  }
}


#undef FM
#undef FA
#undef FS
#undef FMA

}  // namespace bf
