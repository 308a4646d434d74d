// TSDF integration and de-integration on sparse 8x8x8-voxel blocks (Sec. 5.1-5.2).
//
// A voxel keeps integer sums S = sum w d_q, W = sum w and SC = sum w c_q (signed distance
// quantised to 2^-20 m, intensity to 1/65535, w = 1); the paper's running average
// D = (D W + w d) / (W + w) is S 2^-20 / W, and de-integration (the inverse formula) subtracts
// the same integers, so it undoes integration exactly and in any order.
//
// Blocks are found through an open-addressing hash table of packed block coordinates (linear
// probing, insertion by 64-bit compare-and-swap, at most TSDF_MAX_PROBE probes) and live in a
// pool of block records.  One integrate (sign +1) or de-integrate (sign -1) call runs:
//   k_tsdf_touch     one thread per (pixel, band sample): the block containing the sample point
//                    D + k h along the pixel's ray (|k h| <= mu) is looked up or inserted; the
//                    first thread of this call to reach a slot appends it to the touched list
//   k_tsdf_assign    new slots of the touched list get a pool record
//   k_tsdf_integrate one CTA per touched block, one thread per voxel: project the voxel centre,
//                    nearest pixel, d = D - z, skip d < -mu, sdf = min(d, mu), add sign * the
//                    quantised values
// Every floating-point step that decides an integer (a block, a pixel, a quantised value) uses
// explicitly rounded FP32 operations in a fixed order so a CPU restatement takes the same
// decisions; the sums are integers, so the whole volume is bit-for-bit reproducible.
#include "bf_internal.cuh"

namespace bf {

#define FM __fmul_rn
#define FA __fadd_rn
#define FS __fsub_rn

constexpr int TSDF_MAX_PROBE = 256;
constexpr unsigned long long TSDF_EMPTY = ~0ull;

__device__ __forceinline__ unsigned long long tsdf_key(int bx, int by, int bz) {
  return ((unsigned long long)(unsigned)(bx + (1 << 20)) << 42) | ((unsigned long long)(unsigned)(by + (1 << 20)) << 21) |
         (unsigned long long)(unsigned)(bz + (1 << 20));
}

__device__ __forceinline__ unsigned tsdf_hash(unsigned long long k, unsigned mask) {
  return (unsigned)((k * 0x9E3779B97F4A7C15ull) >> 32) & mask;
}

// depth (0 = invalid) and intensity of pixel i of the frame in `slot`
template <int KIND>
__device__ __forceinline__ void load_dc(const FrameStore &fs, long long base, int i, float &d, float &c) {
  if (KIND == BF_STORE_FP32) {
    d = fs.A[base + i].x;
    c = fs.B[base + i].w;
  } else {
    d = __uint_as_float(fs.P16[base + i].x);
    c = f16_to32<KIND>(fs.C16[base + i]);
  }
}

__global__ void k_tsdf_touch(TsdfDev v, FrameStore fs, Intr in, int slot, TsdfPose P, int call_id) {
  const int W = in.W, H = in.H, HW = W * H;
  const int ns = 2 * v.K + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)HW * ns) return;
  const int px = (int)(idx / ns), k = (int)(idx - (long long)px * ns) - v.K;
  float D, C;
  if (fs.storage == BF_STORE_FP32)
    load_dc<BF_STORE_FP32>(fs, (long long)slot * HW, px, D, C);
  else
    D = __uint_as_float(fs.P16[(long long)slot * HW + px].x);
  if (!(D > 0.f)) return;
  const float z = FA(D, FM((float)k, v.h));
  if (!(z > 0.f)) return;
  const int y = px / W, x = px - y * W;
  const float c0 = FM(fs.kx[x], z), c1 = FM(fs.ky[y], z), c2 = z;
  const float p0 = FA(FA(FA(FM(P.R[0], c0), FM(P.R[1], c1)), FM(P.R[2], c2)), P.t[0]);
  const float p1 = FA(FA(FA(FM(P.R[3], c0), FM(P.R[4], c1)), FM(P.R[5], c2)), P.t[1]);
  const float p2 = FA(FA(FA(FM(P.R[6], c0), FM(P.R[7], c1)), FM(P.R[8], c2)), P.t[2]);
  const int bx = (int)floorf(FM(p0, v.inv_block)), by = (int)floorf(FM(p1, v.inv_block)),
            bz = (int)floorf(FM(p2, v.inv_block));
  if (abs(bx) >= (1 << 20) || abs(by) >= (1 << 20) || abs(bz) >= (1 << 20)) {
    atomicOr(v.err, 8);  // outside the addressable range
    return;
  }
  const unsigned long long key = tsdf_key(bx, by, bz);
  unsigned h = tsdf_hash(key, v.mask);
  int found = -1;
  for (int probe = 0; probe < TSDF_MAX_PROBE; ++probe) {
    const unsigned long long cur = ((volatile unsigned long long *)v.keys)[h];
    if (cur == key) {
      found = (int)h;
      break;
    }
    if (cur == TSDF_EMPTY) {
      const unsigned long long old = atomicCAS(v.keys + h, TSDF_EMPTY, key);
      if (old == TSDF_EMPTY || old == key) {
        found = (int)h;
        break;
      }
    }
    h = (h + 1) & v.mask;
  }
  if (found < 0) {
    atomicOr(v.err, 1);  // probe limit: the table is too full
    return;
  }
  if (atomicExch(v.stamp + found, call_id) != call_id) {
    const int i = atomicAdd(v.n_touched, 1);
    if (i < v.max_blocks) v.touched[i] = found;
    else atomicOr(v.err, 4);
  }
}

__global__ void k_tsdf_assign(TsdfDev v) {
  const int n = min(*v.n_touched, v.max_blocks);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int h = v.touched[i];
    if (v.vals[h] >= 0) continue;
    const int b = atomicAdd(v.n_blocks, 1);
    if (b >= v.max_blocks) {
      atomicOr(v.err, 2);  // block pool full
      continue;
    }
    v.vals[h] = b | (1 << 30);  // bit 30: fresh record, zeroed by the integration kernel
  }
}

template <int KIND>
__global__ void __launch_bounds__(512) k_tsdf_integrate(TsdfDev v, FrameStore fs, Intr in, int slot, TsdfPose P,
                                                        int sign) {
  const int W = in.W, H = in.H, HW = W * H;
  const int n = min(*v.n_touched, v.max_blocks);
  const long long base = (long long)slot * HW;
  const int i = threadIdx.x;  // voxel i = ix + 8 iy + 64 iz
  const int ix = i & 7, iy = (i >> 3) & 7, iz = i >> 6;
  for (int e = blockIdx.x; e < n; e += gridDim.x) {
    const int h = v.touched[e];
    const int val = v.vals[h];
    if (val < 0) continue;  // no record (pool full)
    const bool fresh = (val >> 30) & 1;
    const int b = val & ((1 << 30) - 1);
    const unsigned long long key = v.keys[h];
    const int bx = (int)((key >> 42) & 0x1fffff) - (1 << 20), by = (int)((key >> 21) & 0x1fffff) - (1 << 20),
              bz = (int)(key & 0x1fffff) - (1 << 20);
    const float vx = FM(FA((float)(8 * bx + ix), 0.5f), v.vs);
    const float vy = FM(FA((float)(8 * by + iy), 0.5f), v.vs);
    const float vz = FM(FA((float)(8 * bz + iz), 0.5f), v.vs);
    const float d0 = FS(vx, P.t[0]), d1 = FS(vy, P.t[1]), d2 = FS(vz, P.t[2]);
    const float c0 = FA(FA(FM(P.R[0], d0), FM(P.R[3], d1)), FM(P.R[6], d2));  // R^T (v - t)
    const float c1 = FA(FA(FM(P.R[1], d0), FM(P.R[4], d1)), FM(P.R[7], d2));
    const float c2 = FA(FA(FM(P.R[2], d0), FM(P.R[5], d1)), FM(P.R[8], d2));
    int dq = 0, w = 0, cq = 0;
    if (c2 > 0.f) {
      const float iz = __frcp_rn(c2);
      const float ux = FA(FM(in.fx, FM(c0, iz)), in.cx), uy = FA(FM(in.fy, FM(c1, iz)), in.cy);
      const float pxf = floorf(FA(ux, 0.5f)), pyf = floorf(FA(uy, 0.5f));
      if (pxf >= 0.f && pxf <= (float)(W - 1) && pyf >= 0.f && pyf <= (float)(H - 1)) {
        float D, C;
        load_dc<KIND>(fs, base, (int)pyf * W + (int)pxf, D, C);
        if (D > 0.f) {
          const float sd = FS(D, c2);
          if (sd >= -v.mu) {
            const float sdf = fminf(sd, v.mu);
            dq = __float2int_rn(FM(sdf, v.inv_q));
            cq = __float2int_rn(FM(C, 65535.f));
            w = 1;
          }
        }
      }
    }
    int *S = v.S + (long long)b * 512, *Wt = v.W + (long long)b * 512, *SC = v.SC + (long long)b * 512;
    const int s0 = fresh ? 0 : S[i], w0 = fresh ? 0 : Wt[i], c0q = fresh ? 0 : SC[i];
    S[i] = s0 + sign * dq;
    Wt[i] = w0 + sign * w;
    SC[i] = c0q + sign * cq;
    __syncthreads();
    if (i == 0 && fresh) v.vals[h] = b;  // the record now holds valid sums
  }
}

int launch_tsdf(const TsdfDev &v, const FrameStore &fs, const Intr &in, int slot, const TsdfPose &P, int sign,
                int call_id, cudaStream_t st) {
  const long long n = (long long)in.W * in.H * (2 * v.K + 1);
  cudaMemsetAsync(v.n_touched, 0, sizeof(int), st);
  k_tsdf_touch<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, fs, in, slot, P, call_id);
  k_tsdf_assign<<<148, 256, 0, st>>>(v);
  if (fs.storage == BF_STORE_BF16)
    k_tsdf_integrate<BF_STORE_BF16><<<4 * 148, 512, 0, st>>>(v, fs, in, slot, P, sign);
  else if (fs.storage == BF_STORE_FP16)
    k_tsdf_integrate<BF_STORE_FP16><<<4 * 148, 512, 0, st>>>(v, fs, in, slot, P, sign);
  else
    k_tsdf_integrate<BF_STORE_FP32><<<4 * 148, 512, 0, st>>>(v, fs, in, slot, P, sign);
  return 3;
}

}  // namespace bf
