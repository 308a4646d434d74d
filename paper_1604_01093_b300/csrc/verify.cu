// Dense two-sided verification of frame pairs (Sec. 4.1.1), also used for chunk validation
// (Sec. 4.2).
//
// The paper runs it as a single kernel in which each thread block handles one pair of images and
// the re-projection error is formed by local reductions; so does this one.  For each direction
// (i -> j with T_ij, then j -> i with T_ji) every source pixel with valid depth and normal is
// projected into the other frame and matched to the nearest pixel; the match is kept when the
// distance, normal and photoconsistency gates pass:
//   ||T p - q|| < tau_d,  (R n_src) . n_dst > tau_n,  |C_src(x, y) - C_dst(target)| < tau_c.
// The CTA counts the kept matches and sums their distances per direction.
//
// The gate decisions use explicitly rounded FP32 operations in a fixed order; they agree with the
// exact (FP64) test except where a value lies within FP32 rounding of its threshold.
#include "bf_internal.cuh"

namespace bf {

#define FM __fmul_rn
#define FA __fadd_rn
#define FS __fsub_rn

constexpr int VERIFY_BS = 256;

// (D, n) and intensity of pixel i of the frame in `slot`
template <int KIND>
__device__ __forceinline__ void load_dnc(const FrameStore &fs, long long base, int i, float4 &dn, float &c) {
  if (KIND == BF_STORE_FP32) {
    dn = fs.A[base + i];
    c = fs.B[base + i].w;
  } else {
    dn = unpack16_dn<KIND>(fs.P16[base + i]);
    c = f16_to32<KIND>(fs.C16[base + i]);
  }
}

template <int KIND>
__global__ void __launch_bounds__(VERIFY_BS)
    k_verify(const VerifyPair *__restrict__ rec, FrameStore fs, Intr in, float tau_d2, float tau_n, float tau_c,
             double *__restrict__ out) {
  __shared__ float ktab[2 * 1024];
  __shared__ double wsum[2][VERIFY_BS / 32];
  __shared__ int wcnt[2][VERIFY_BS / 32];
  const int W = in.W, H = in.H, HW = W * H;
  const VerifyPair &P = rec[blockIdx.x];
  const bool tab = W + H <= 2 * 1024;
  const float *kx = fs.kx, *ky = fs.ky;
  if (tab) {
    for (int k = threadIdx.x; k < W + H; k += VERIFY_BS) ktab[k] = k < W ? fs.kx[k] : fs.ky[k - W];
    kx = ktab;
    ky = ktab + W;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const long long sb = (long long)(dir == 0 ? P.slot_i : P.slot_j) * HW;
    const long long tb = (long long)(dir == 0 ? P.slot_j : P.slot_i) * HW;
    const float *M = P.M[dir];
    const float R00 = M[0], R01 = M[1], R02 = M[2], R10 = M[3], R11 = M[4], R12 = M[5], R20 = M[6], R21 = M[7],
                R22 = M[8], t0 = M[9], t1 = M[10], t2 = M[11];
    int cnt = 0;
    float sum = 0.f;
    for (int px = threadIdx.x; px < HW; px += VERIFY_BS) {
      float4 a;
      float ca;
      load_dnc<KIND>(fs, sb, px, a, ca);
      const bool nvalid = (a.y != 0.f) || (a.z != 0.f) || (a.w != 0.f);
      if (!(a.x > 0.f && nvalid)) continue;
      const int y = px / W, x = px - y * W;
      const float z = a.x;
      const float dx = FM(kx[x], z), dy = FM(ky[y], z), dz = z;
      const float Y0 = FA(FA(FA(FM(R00, dx), FM(R01, dy)), FM(R02, dz)), t0);
      const float Y1 = FA(FA(FA(FM(R10, dx), FM(R11, dy)), FM(R12, dz)), t1);
      const float Y2 = FA(FA(FA(FM(R20, dx), FM(R21, dy)), FM(R22, dz)), t2);
      if (!(Y2 > 0.f)) continue;
      const float iz = __frcp_rn(Y2);
      const float ux = FA(FM(in.fx, FM(Y0, iz)), in.cx);
      const float uy = FA(FM(in.fy, FM(Y1, iz)), in.cy);
      const float nxf = floorf(FA(ux, 0.5f)), nyf = floorf(FA(uy, 0.5f));
      if (!(nxf >= 0.f && nxf <= (float)(W - 1) && nyf >= 0.f && nyf <= (float)(H - 1))) continue;
      const int tx = (int)nxf, ty = (int)nyf;
      float4 b;
      float cb;
      load_dnc<KIND>(fs, tb, ty * W + tx, b, cb);
      const bool tnvalid = (b.y != 0.f) || (b.z != 0.f) || (b.w != 0.f);
      if (!(b.x > 0.f && tnvalid)) continue;
      const float qx = FM(kx[tx], b.x), qy = FM(ky[ty], b.x), qz = b.x;
      const float ex = FS(Y0, qx), ey = FS(Y1, qy), ez = FS(Y2, qz);
      const float dist2 = FA(FA(FM(ex, ex), FM(ey, ey)), FM(ez, ez));
      const float m0 = FA(FA(FM(R00, a.y), FM(R01, a.z)), FM(R02, a.w));
      const float m1 = FA(FA(FM(R10, a.y), FM(R11, a.z)), FM(R12, a.w));
      const float m2 = FA(FA(FM(R20, a.y), FM(R21, a.z)), FM(R22, a.w));
      const float ndot = FA(FA(FM(m0, b.y), FM(m1, b.z)), FM(m2, b.w));
      if (!(dist2 < tau_d2 && ndot > tau_n && fabsf(FS(ca, cb)) < tau_c)) continue;
      ++cnt;
      sum += sqrtf(dist2);
    }
    // fixed-order reduction: FP32 warp trees, warps summed in FP64 in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (lane == 0) {
      wcnt[dir][warp] = cnt;
      wsum[dir][warp] = (double)sum;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int dir = threadIdx.x;
    long long n = 0;
    double e = 0.0;
    for (int w = 0; w < VERIFY_BS / 32; ++w) {
      n += wcnt[dir][w];
      e += wsum[dir][w];
    }
    out[4 * blockIdx.x + dir] = (double)n;
    out[4 * blockIdx.x + 2 + dir] = e;
  }
}

int launch_verify(int n_pairs, const VerifyPair *rec, const FrameStore &fs, const Intr &in, float tau_d2,
                  float tau_n, float tau_c, double *out, cudaStream_t st) {
  if (n_pairs <= 0) return 0;
  if (fs.storage == BF_STORE_BF16)
    k_verify<BF_STORE_BF16><<<n_pairs, VERIFY_BS, 0, st>>>(rec, fs, in, tau_d2, tau_n, tau_c, out);
  else if (fs.storage == BF_STORE_FP16)
    k_verify<BF_STORE_FP16><<<n_pairs, VERIFY_BS, 0, st>>>(rec, fs, in, tau_d2, tau_n, tau_c, out);
  else
    k_verify<BF_STORE_FP32><<<n_pairs, VERIFY_BS, 0, st>>>(rec, fs, in, tau_d2, tau_n, tau_c, out);
  return 1;
}

}  // namespace bf
