// Per-frame preprocessing and correspondence packing.
//
// Sec. 4.1.1 caches per frame the low-resolution depth with its camera-space positions and
// normals; Sec. 4.3 evaluates the photometric term on I, the gradient of the luminance.
// Readings (no formulas in the paper): depth valid iff finite and depth_min < D < depth_max;
// normal = normalize((P(x,y+1)-P(x,y-1)) x (P(x+1,y)-P(x-1,y))), valid on the 1-pixel interior
// when the pixel and its 4 neighbours are valid and the cross product's norm >= 1e-12;
// I = |grad L| by central differences on the 1-pixel interior; grad I by central differences
// of I on the 2-pixel interior.
#include "bf_internal.cuh"

namespace bf {

__device__ __forceinline__ bool depth_ok(float z, float dmin, float dmax) {
  return isfinite(z) && z > dmin && z < dmax;
}

// |grad L| at interior pixel pix (central differences).
__device__ __forceinline__ float lum_grad_mag(const float *__restrict__ Lf, int pix, int W) {
  const float gx = 0.5f * (Lf[pix + 1] - Lf[pix - 1]);
  const float gy = 0.5f * (Lf[pix + W] - Lf[pix - W]);
  return sqrtf(gx * gx + gy * gy);
}

// Depth (0 if invalid) and unit normal (0 if invalid) of pixel (x, y).
__device__ __forceinline__ float4 depth_normal(const float *__restrict__ Df, int pix, int x, int y,
                                               const FrameStore &fs, float dmin, float dmax) {
  const int W = fs.W, H = fs.H;
  const float z = Df[pix];
  const bool ok = depth_ok(z, dmin, dmax);
  float4 a = make_float4(ok ? z : 0.f, 0.f, 0.f, 0.f);
  if (ok && x >= 1 && x <= W - 2 && y >= 1 && y <= H - 2) {
    const float zl = Df[pix - 1], zr = Df[pix + 1], zu = Df[pix - W], zd = Df[pix + W];
    if (depth_ok(zl, dmin, dmax) && depth_ok(zr, dmin, dmax) && depth_ok(zu, dmin, dmax) &&
        depth_ok(zd, dmin, dmax)) {
      const float kxl = fs.kx[x - 1], kxr = fs.kx[x + 1], kxc = fs.kx[x];
      const float kyu = fs.ky[y - 1], kyd = fs.ky[y + 1], kyc = fs.ky[y];
      // dy = P(x,y+1) - P(x,y-1), dx = P(x+1,y) - P(x-1,y)
      const float dyx = kxc * zd - kxc * zu, dyy = kyd * zd - kyu * zu, dyz = zd - zu;
      const float dxx = kxr * zr - kxl * zl, dxy = kyc * zr - kyc * zl, dxz = zr - zl;
      const float cx = dyy * dxz - dyz * dxy;
      const float cy = dyz * dxx - dyx * dxz;
      const float cz = dyx * dxy - dyy * dxx;
      const float nrm = sqrtf(cx * cx + cy * cy + cz * cz);
      if (nrm >= 1e-12f) {
        a.y = cx / nrm;
        a.z = cy / nrm;
        a.w = cz / nrm;
      }
    }
  }
  return a;
}

// FP32 storage, one pass (one thread per pixel of n frames): (D, n) into A and (I, grad I, L)
// into B.  grad I on the 2-pixel interior from the neighbours' I recomputed from the luminance
// (the same function as the pixel's own I, so the same values a second pass over the stored I
// would read); one read of depth and luminance and one write of A and B per pixel.
__global__ void k_pre32(const float *__restrict__ depth, const float *__restrict__ lum, int n,
                        const int *__restrict__ slots, FrameStore fs, float4 *__restrict__ A,
                        float4 *__restrict__ B, float dmin, float dmax) {
  const int W = fs.W, H = fs.H;
  const long long HW = (long long)W * H;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * HW) return;
  const int f = (int)(idx / HW);
  const int pix = (int)(idx - (long long)f * HW);
  const int y = pix / W, x = pix - y * W;
  const float *Df = depth + (long long)f * HW;
  const float *Lf = lum + (long long)f * HW;
  const float4 a = depth_normal(Df, pix, x, y, fs, dmin, dmax);
  float I = 0.f, Ix = 0.f, Iy = 0.f;
  if (x >= 1 && x <= W - 2 && y >= 1 && y <= H - 2) I = lum_grad_mag(Lf, pix, W);
  if (x >= 2 && x <= W - 3 && y >= 2 && y <= H - 3) {
    Ix = 0.5f * (lum_grad_mag(Lf, pix + 1, W) - lum_grad_mag(Lf, pix - 1, W));
    Iy = 0.5f * (lum_grad_mag(Lf, pix + W, W) - lum_grad_mag(Lf, pix - W, W));
  }
  const long long o = (long long)slots[f] * HW + pix;
  A[o] = a;
  B[o] = make_float4(I, Ix, Iy, Lf[pix]);  // w: the intensity itself (dense verification)
}

// 16-bit storage: one pass writes the packed record (depth FP32, normal, I, grad I rounded to
// BF16 / FP16); the neighbours' I for grad I is recomputed from the luminance in FP32, so grad I
// is formed from unrounded I exactly as in the FP32 path and rounded once.
template <int KIND>
__global__ void k_pre16(const float *__restrict__ depth, const float *__restrict__ lum, int n,
                        const int *__restrict__ slots, FrameStore fs, uint4 *__restrict__ P,
                        unsigned short *__restrict__ C16, float dmin, float dmax) {
  const int W = fs.W, H = fs.H;
  const long long HW = (long long)W * H;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * HW) return;
  const int f = (int)(idx / HW);
  const int pix = (int)(idx - (long long)f * HW);
  const int y = pix / W, x = pix - y * W;
  const float *Df = depth + (long long)f * HW;
  const float *Lf = lum + (long long)f * HW;
  const float4 a = depth_normal(Df, pix, x, y, fs, dmin, dmax);
  float I = 0.f, Ix = 0.f, Iy = 0.f;
  if (x >= 1 && x <= W - 2 && y >= 1 && y <= H - 2) I = lum_grad_mag(Lf, pix, W);
  if (x >= 2 && x <= W - 3 && y >= 2 && y <= H - 3) {
    Ix = 0.5f * (lum_grad_mag(Lf, pix + 1, W) - lum_grad_mag(Lf, pix - 1, W));
    Iy = 0.5f * (lum_grad_mag(Lf, pix + W, W) - lum_grad_mag(Lf, pix - W, W));
  }
  const long long o = (long long)slots[f] * HW + pix;
  P[o] = pack16<KIND>(a, I, Ix, Iy);
  C16[o] = f32_to16<KIND>(Lf[pix]);
}

int launch_preprocess(const float *depth, const float *lum, int n, const int *slots_dev, FrameStore fs,
                       float4 *A, float4 *B, uint4 *P16, unsigned short *C16, float dmin, float dmax,
                       cudaStream_t st) {
  const long long total = (long long)n * fs.W * fs.H;
  if (total == 0) return 0;
  const int bs = 256;
  const unsigned grid = (unsigned)((total + bs - 1) / bs);
  if (fs.storage == BF_STORE_BF16) {
    k_pre16<BF_STORE_BF16><<<grid, bs, 0, st>>>(depth, lum, n, slots_dev, fs, P16, C16, dmin, dmax);
    return 1;
  }
  if (fs.storage == BF_STORE_FP16) {
    k_pre16<BF_STORE_FP16><<<grid, bs, 0, st>>>(depth, lum, n, slots_dev, fs, P16, C16, dmin, dmax);
    return 1;
  }
  k_pre32<<<grid, bs, 0, st>>>(depth, lum, n, slots_dev, fs, A, B, dmin, dmax);
  return 1;
}

// Correspondences into the pool as (p, w) / (q, 0) float4 pairs; swap exchanges p and q so that
// p always belongs to the smaller frame id.
__global__ void k_pack_corr(const float *__restrict__ p_i, const float *__restrict__ p_j,
                            const float *__restrict__ w, int n, int swap, float4 *__restrict__ P,
                            float4 *__restrict__ Q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float *a = swap ? p_j : p_i;
  const float *b = swap ? p_i : p_j;
  P[k] = make_float4(a[3 * k], a[3 * k + 1], a[3 * k + 2], w ? w[k] : 1.f);
  Q[k] = make_float4(b[3 * k], b[3 * k + 1], b[3 * k + 2], 0.f);
}

int launch_pack_corr(const float *p_i, const float *p_j, const float *w, int n, int swap, float4 *P, float4 *Q,
                      cudaStream_t st) {
  if (n <= 0) return 0;
  k_pack_corr<<<(n + 255) / 256, 256, 0, st>>>(p_i, p_j, w, n, swap, P, Q);
  return 1;
}

// Batched variant: correspondence k belongs to the pair whose [off[p], off[p+1]) holds it
// (binary search over n_pairs + 1 offsets); swap[p] as above.
__global__ void k_pack_corr_batch(const float *__restrict__ p_i, const float *__restrict__ p_j,
                                  const float *__restrict__ w, int n_total, const int *__restrict__ off,
                                  const int *__restrict__ swap, int n_pairs, float4 *__restrict__ P,
                                  float4 *__restrict__ Q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_total) return;
  int lo = 0, hi = n_pairs - 1;  // largest p with off[p] <= k
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  const bool s = swap[lo] != 0;
  const float *a = s ? p_j : p_i;
  const float *b = s ? p_i : p_j;
  P[k] = make_float4(a[3 * k], a[3 * k + 1], a[3 * k + 2], w ? w[k] : 1.f);
  Q[k] = make_float4(b[3 * k], b[3 * k + 1], b[3 * k + 2], 0.f);
}

int launch_pack_corr_batch(const float *p_i, const float *p_j, const float *w, int n_total, const int *off,
                           const int *swap, int n_pairs, float4 *P, float4 *Q, cudaStream_t st) {
  if (n_total <= 0 || n_pairs <= 0) return 0;
  k_pack_corr_batch<<<(n_total + 255) / 256, 256, 0, st>>>(p_i, p_j, w, n_total, off, swap, n_pairs, P, Q);
  return 1;
}

}  // namespace bf
