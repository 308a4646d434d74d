// Persistent batched solve: the whole Gauss-Newton loop of a batch of independent problems
// (chunks, Sec. 4.2) in ONE kernel launch.
//
// The launch is cooperative (every CTA resident) and its CTAs take work items from a device
// queue in publication order.  An item is one of
//   XFORM(p)          pair transforms of problem p at its initial poses
//   DENSE(p, g, k)    dense tile k of p at Gauss-Newton iteration g (ACCUM partial sums)
//   SPARSE(p, g, s)   correspondence segment s of p at iteration g
//   SOLVE(p, g)       p's pair merge, frame assembly, PCG, energy record, pose update and
//                     pair transforms for iteration g + 1
//   EDENSE / ESPARSE  the final energy evaluation's tiles / segments (r_max)
//   FINAL(p)          p's merge of those and its final energy record
// The code of every item is the device function the launch-sequence path runs (dense_tile,
// sparse_seg, merge_pair, assemble_var, pcg_problem), so a problem gets the same bits either
// way, alone or inside any batch.  Completing an item publishes what it unblocks: the CTA
// finishing the last tile or segment of (p, g) publishes SOLVE(p, g); SOLVE(p, g) publishes
// p's tiles and segments of iteration g + 1.  Problems therefore advance independently: a
// 3-frame chunk runs its later iterations while an 11-frame chunk still evaluates tiles, and
// one problem's solve overlaps the other problems' dense work instead of waiting for a kernel
// boundary.
//
// Deadlock freedom: a CTA claims slot h only after every slot before h has been claimed, and a
// slot is claimed only once published, so every item in progress belongs to a running CTA and
// whatever it unblocks is published when it ends.  Every wait (for a slot to be published) is
// bounded; a CTA that gives up sets the queue's error word, every waiting CTA then leaves, and
// the host reports BF_ERR_TIMEOUT.
//
// Data written by one CTA and read by another (pair transforms, poses, partial sums) is read
// through L2 (the CG variants of the item functions): an SM's L1 may still hold the copy of an
// earlier Gauss-Newton iteration.
#include "dense_eval.cuh"
#include "solve_eval.cuh"
#include "sparse_eval.cuh"

namespace bf {

enum : int { IT_XFORM = 0, IT_DENSE = 1, IT_SPARSE = 2, IT_SOLVE = 3, IT_EDENSE = 4, IT_ESPARSE = 5, IT_FINAL = 6 };

constexpr int BATCH_BS = 256;  // = DENSE_BS = PCG_BS
static_assert(BATCH_BS == DENSE_BS && BATCH_BS == PCG_BS && BATCH_BS >= SPARSE_BS, "one CTA shape for all items");
// Polls of a slot's flag before a CTA gives up: the first 2^10 back to back, then with a 256 ns
// back-off, about 4 s in all (a legitimate wait ends when an item in progress on another CTA
// finishes and publishes its followers: milliseconds at most).
constexpr long long BATCH_WAIT_LIMIT = 1LL << 24;

// Shared memory of one CTA: the item functions' scratch, one at a time.
template <typename Acc>
struct BatchSmem {
  union {
    float dred[DENSE_BS / 32][NPD];
    struct {
      MergeSmem<Acc> m[BATCH_BS / 32];
      AsmSmem a[BATCH_BS / 32];
    } ma;
    PcgSmem<Acc> pcg;
  } u;
  int4 item;
  int stop, base;
  BatchArgs args;   // this CTA's copy of the kernel arguments, read by the out-of-line item handlers
  BatchQueue queue;
};

// Publish the items of problem p's stage g (g < n_gn: its tiles and segments of iteration g;
// g == n_gn: the final energy's); a problem without any goes straight to SOLVE / FINAL.  Called
// by every thread of the CTA.
template <typename Acc>
__device__ void publish_stage(const BatchArgs &a, const BatchQueue &q, int p, int g, BatchSmem<Acc> &sm) {
  const Tables &t = a.t;
  const int tile0 = t.prob_tile0[p], nt = t.prob_tile1[p] - tile0;
  const int seg0 = t.prob_seg0[p], ns = t.prob_seg1[p] - seg0;
  const bool fin = g == a.n_gn;
  const int n = nt + ns > 0 ? nt + ns : 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int base = q.n_prob + atomicAdd(q.tail, n);
    if (base + n > q.total) atomicExch(q.err, 2);  // cannot happen with consistent tables
    sm.base = base;
  }
  __syncthreads();
  const int base = sm.base;
  if (base + n > q.total) return;
  for (int k = threadIdx.x; k < n; k += BATCH_BS) {
    int4 it;
    if (nt + ns == 0)
      it = make_int4(fin ? IT_FINAL : IT_SOLVE, p, g, 0);
    else if (k < nt)
      it = make_int4(fin ? IT_EDENSE : IT_DENSE, p, g, tile0 + k);
    else
      it = make_int4(fin ? IT_ESPARSE : IT_SPARSE, p, g, seg0 + k - nt);
    __stcg(q.items + base + k, it);
    __threadfence();
    *(volatile int *)(q.flags + base + k) = 1;
  }
}

// After a tile / segment item: count it; the CTA that completes the stage publishes its follower.
template <typename Acc>
__device__ void finish_part(const BatchArgs &a, const BatchQueue &q, int p, int g, bool fin, BatchSmem<Acc> &sm) {
  __threadfence();  // this CTA's partial record before the count
  __syncthreads();
  if (threadIdx.x == 0) {
    const Tables &t = a.t;
    const int n = (t.prob_tile1[p] - t.prob_tile0[p]) + (t.prob_seg1[p] - t.prob_seg0[p]);
    const int c = atomicAdd(q.done + p, 1) + 1;
    if (c == n) {
      q.done[p] = 0;  // no other item of p is in flight until the next stage is published
      const int slot = q.n_prob + atomicAdd(q.tail, 1);
      if (slot >= q.total) {
        atomicExch(q.err, 2);
      } else {
        __stcg(q.items + slot, make_int4(fin ? IT_FINAL : IT_SOLVE, p, g, 0));
        __threadfence();
        *(volatile int *)(q.flags + slot) = 1;
      }
    }
  }
}

template <typename Acc>
__device__ void merge_problem(const BatchArgs &a, int p, BatchSmem<Acc> &sm) {
  const Tables &t = a.t;
  const int warp = threadIdx.x >> 5;
  for (int pr = t.prob_pair0[p] + warp; pr < t.prob_pair1[p]; pr += BATCH_BS / 32)
    merge_pair<Acc, Acc, true>(pr, t, a.pose, (const Acc *)a.dpart, (const Acc *)a.spart, (Acc *)a.pairblk,
                               (Acc *)a.pairen, a.pairoff, sm.u.ma.m[warp]);
  __syncthreads();
}

// Item handlers.  All but the dense tile are compiled on their own (not inlined into the dispatch
// loop), so the loop's register allocation is the dense tile's, as in k_dense.
// The count after a dense tile, out of line: the item is read back from shared memory, so that
// nothing of it stays live in registers across the tile's pixel loop (fewer spills there).
template <typename Acc>
__device__ __noinline__ void item_dense_done(const BatchArgs &a, const BatchQueue &q, BatchSmem<Acc> &sm) {
  volatile int *vi = (volatile int *)&sm.item;
  const int4 it = make_int4(vi[0], vi[1], vi[2], vi[3]);
  finish_part<Acc>(a, q, it.y, it.z, it.x == IT_EDENSE, sm);
}

template <typename Acc, int KIND>
__device__ __forceinline__ void item_dense(const BatchArgs &a, const BatchQueue &q, int4 it, float *ktab,
                                        BatchSmem<Acc> &sm) {
  const bool fin = it.x == IT_EDENSE;
  if (fin)
    dense_tile<MODE_ENERGY, KIND, Acc, true>(it.w, a.t, a.fs, a.in, a.pairM, a.gates, a.wg[a.n_gn], a.wp[a.n_gn],
                                             (Acc *)a.dpart, nullptr, ktab, sm.u.dred);
  else
    dense_tile<MODE_ACCUM, KIND, Acc, true>(it.w, a.t, a.fs, a.in, a.pairM, a.gates, a.wg[it.z], a.wp[it.z],
                                            (Acc *)a.dpart, nullptr, ktab, sm.u.dred);
  item_dense_done<Acc>(sm.args, sm.queue, sm);
}

template <typename Acc>
__device__ __noinline__ void item_sparse(const BatchArgs &a, const BatchQueue &q, int4 it, BatchSmem<Acc> &sm) {
  const bool fin = it.x == IT_ESPARSE;
  if (threadIdx.x < 32) {  // one warp per segment, as k_sparse
    if (fin)
      sparse_seg<MODE_ENERGY, Acc, true>(it.w, a.t, a.P, a.Q, a.pairM, a.w_sparse, (Acc *)a.spart, a.srmax, a.srarg);
    else
      sparse_seg<MODE_ACCUM, Acc, true>(it.w, a.t, a.P, a.Q, a.pairM, a.w_sparse, (Acc *)a.spart, a.srmax, a.srarg);
  }
  finish_part<Acc>(a, q, it.y, it.z, fin, sm);
}

template <typename Acc>
__device__ __noinline__ void item_xform(const BatchArgs &a, const BatchQueue &q, int p, BatchSmem<Acc> &sm) {
  const Tables &t = a.t;
  // one thread per transform entry (24 per pair), like k_pair_xform
  const int p0 = t.prob_pair0[p], n = 24 * (t.prob_pair1[p] - p0);
  for (int k = threadIdx.x; k < n; k += BATCH_BS) {
    const int pr = p0 + k / 24, e = k % 24;
    double Ta[12], Tb[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      Ta[m] = __ldcg(a.pose + 12 * t.pair_a[pr] + m);
      Tb[m] = __ldcg(a.pose + 12 * t.pair_b[pr] + m);
    }
    a.pairM[24 * pr + e] = e < 12 ? pair_xform_entry(Ta, Tb, e) : pair_xform_entry(Tb, Ta, e - 12);
  }
  publish_stage<Acc>(a, q, p, 0, sm);  // stage 0 is the final energy when n_gn = 0
}

template <typename Acc>
__device__ __noinline__ void item_solve(const BatchArgs &a, const BatchQueue &q, int p, int g, BatchSmem<Acc> &sm) {
  const Tables &t = a.t;
  merge_problem<Acc>(a, p, sm);
  const int warp = threadIdx.x >> 5;
  for (int v = t.prob_var0[p] + warp; v < t.prob_var1[p]; v += BATCH_BS / 32)
    assemble_var<Acc>(v, t, (const Acc *)a.pairblk, a.precond, (Acc *)a.Dd, (Acc *)a.rhs, a.Df, a.Minv, a.vflags,
                      sm.u.ma.a[warp]);
  __syncthreads();
  PcgOut po;
  po.energy = a.energy + (size_t)g * t.n_prob * PAIREN;
  po.pose = a.pose;
  po.pairM = a.pairM;
  MatFree mf{};
  pcg_problem<Acc, true>(p, t, a.Df, a.pairoff, a.Minv, (const Acc *)a.rhs, a.x, a.r, a.z, a.p, a.q, a.n_pcg,
                         a.pflags, (const Acc *)a.pairen, po, mf, sm.u.pcg);
  publish_stage<Acc>(a, q, p, g + 1, sm);
}

template <typename Acc>
__device__ __noinline__ void item_final(const BatchArgs &a, int p, BatchSmem<Acc> &sm) {
  merge_problem<Acc>(a, p, sm);
  problem_energy<Acc>(a.t, (const Acc *)a.pairen, p, a.energy + (size_t)a.n_gn * a.t.n_prob * PAIREN, sm.u.pcg.esh);
}

// Three CTAs per SM (up to 85 registers per thread): with four (64 registers, as k_dense has)
// the dense tile's pixel loop spills inside this kernel and runs 1.8x slower per tile; with three
// it does not spill and runs 17 % below k_dense's per-SM rate (fewer warps to hide latency).
template <typename Acc, int KIND>
__global__ void __launch_bounds__(BATCH_BS, 3) k_batch(BatchArgs a, BatchQueue q) {
  extern __shared__ float ktab[];  // kx[W], ky[H]
  __shared__ BatchSmem<Acc> sm;
  // the out-of-line handlers read the arguments from shared memory, so the parameter block is
  // never copied to local memory and the inlined dense path reads it as k_dense does
  {
    const int *src = (const int *)&a;
    int *dst = (int *)&sm.args;
    for (int k = threadIdx.x; k < (int)(sizeof(BatchArgs) / sizeof(int)); k += BATCH_BS) dst[k] = src[k];
    const int *qs = (const int *)&q;
    int *qd = (int *)&sm.queue;
    for (int k = threadIdx.x; k < (int)(sizeof(BatchQueue) / sizeof(int)); k += BATCH_BS) qd[k] = qs[k];
  }
  for (;;) {
    if (threadIdx.x == 0) {
      int stop = 0;
      int4 it = make_int4(0, 0, 0, 0);
      const int h = atomicAdd(q.head, 1);
      if (h >= q.total) {
        stop = 1;
      } else if (h < q.n_prob) {
        it = make_int4(IT_XFORM, h, 0, 0);  // the first n_prob slots are implicit
      } else if (!wait_published(q.flags + h, q.err, q.wait_limit)) {
        atomicCAS(q.err, 0, 1);
        stop = 1;
      } else {
        __threadfence();
        it = __ldcg(q.items + h);
      }
      sm.stop = stop;
      sm.item = it;
    }
    __syncthreads();
    if (sm.stop) break;
    const int4 it = sm.item;
    switch (it.x) {
      case IT_XFORM:
        item_xform<Acc>(sm.args, sm.queue, it.y, sm);
        break;
      case IT_DENSE:
      case IT_EDENSE:
        item_dense<Acc, KIND>(a, q, it, ktab, sm);
        break;
      case IT_SPARSE:
      case IT_ESPARSE:
        item_sparse<Acc>(sm.args, sm.queue, it, sm);
        break;
      case IT_SOLVE:
        item_solve<Acc>(sm.args, sm.queue, it.y, it.z, sm);
        break;
      case IT_FINAL:
        item_final<Acc>(sm.args, it.y, sm);
        break;
      default:
        break;
    }
    __syncthreads();
  }
}

template <typename Acc, int KIND>
static int batch_grid(size_t smem) {
  static PerDevice blocks;  // one per instantiation, per device and dynamic shared memory size
  return (int)blocks.get((long long)smem, [smem] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<Acc, KIND>, BATCH_BS, smem) != cudaSuccess) {
      per_sm = 0;
      cudaGetLastError();
    }
    return (long long)sms * per_sm;
  });
}

template <typename Acc, int KIND>
static int batch_go(const BatchArgs &a, const BatchQueue &q, cudaStream_t st) {
  const size_t smem = (size_t)(a.in.W + a.in.H) * sizeof(float);
  const int grid = batch_grid<Acc, KIND>(smem);
  if (grid <= 0) return -1;
  BatchArgs aa = a;
  BatchQueue qq = q;
  void *args[] = {&aa, &qq};
  if (cudaLaunchCooperativeKernel((const void *)k_batch<Acc, KIND>, dim3(grid), dim3(BATCH_BS), args, smem, st) !=
      cudaSuccess)
    return -1;
  return 1;
}

template <typename Acc>
int launch_batch(const BatchArgs &a, void *qmem, long long total, cudaStream_t st) {
  const int n_prob = a.t.n_prob;
  if (n_prob == 0) return 0;
  char *m = (char *)qmem;
  BatchQueue q;
  q.head = (int *)m;
  q.tail = (int *)(m + 4);
  q.err = (int *)(m + 8);
  q.done = (int *)(m + 256);
  q.flags = (int *)(m + 256 + 4 * (size_t)n_prob);
  const size_t zero_bytes = batch_zero_bytes(n_prob, total);
  q.items = (int4 *)(m + zero_bytes);
  q.n_prob = n_prob;
  q.total = (int)total;
  q.wait_limit = BATCH_WAIT_LIMIT;
  // counters, completion counts and publication flags start at zero (tail counts published slots
  // beyond the n_prob implicit XFORM items)
  if (cudaMemsetAsync(m, 0, zero_bytes, st) != cudaSuccess) return -1;
  if (a.fs.storage == BF_STORE_BF16) return batch_go<Acc, BF_STORE_BF16>(a, q, st);
  if (a.fs.storage == BF_STORE_FP16) return batch_go<Acc, BF_STORE_FP16>(a, q, st);
  return batch_go<Acc, BF_STORE_FP32>(a, q, st);
}
template int launch_batch<double>(const BatchArgs &, void *, long long, cudaStream_t);
template int launch_batch<float>(const BatchArgs &, void *, long long, cudaStream_t);

}  // namespace bf
