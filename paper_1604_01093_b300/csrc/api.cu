// C ABI of the library: context, frame store, correspondence pool, solve orchestration.
//
// A solve (local, batched local or global) is flattened into one set of tables: frames of
// all its problems, unordered pairs with correspondences, directed dense pairs split into
// pixel tiles, correspondence segments, and per-frame incidence lists.  The Gauss-Newton loop
// then runs on the context's stream as a fixed sequence of kernels per iteration
// (Sec. 4.4: linearise, assemble J^T J and -J^T F, PCG, update), with the energy evaluated
// before each step and after the last one.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <map>
#include <mutex>
#include <thread>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "bf_internal.cuh"
#include "bf.h"

using namespace bf;

namespace {

struct FrameInfo {
  int slot = -1;
  bool has_world = false;
  double world[12];      // R row-major, t
  int member_of = -1;    // chunk whose non-first member this frame is (latest local solve)
  int keyframe_of = -1;  // chunk whose first frame this frame is
};

struct Chunk {
  std::vector<int> frames;
  std::vector<std::array<double, 12>> local;  // pose relative to frames[0]
};

struct Seg {
  int off, cnt;
};

typedef std::array<double, 12> Pose12;

Pose12 ident12() { return Pose12{1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0}; }

Pose12 from16(const double *m) {
  return Pose12{m[0], m[1], m[2], m[4], m[5], m[6], m[8], m[9], m[10], m[3], m[7], m[11]};
}
void to16(const Pose12 &p, double *m) {
  const double v[16] = {p[0], p[1], p[2], p[9], p[3], p[4], p[5], p[10], p[6], p[7], p[8], p[11], 0, 0, 0, 1};
  std::memcpy(m, v, sizeof(v));
}
Pose12 compose(const Pose12 &A, const Pose12 &B) {  // A * B
  Pose12 C;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    C[9 + i] = A[3 * i] * B[9] + A[3 * i + 1] * B[10] + A[3 * i + 2] * B[11] + A[9 + i];
  }
  return C;
}

inline uint64_t pair_key(int a, int b) {
  const uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
  return ((uint64_t)lo << 32) | hi;
}

}  // namespace

// Everything one solve in flight needs besides the shared frame store and correspondence pool:
// a stream, the workspace arena, pinned staging and the cached Gauss-Newton graph.
namespace {
struct TableCache;  // defined with the solve tables below
}

struct Exec {
  cudaStream_t st = nullptr;
  cudaStream_t st_hi = nullptr, st_lo = nullptr;  // serving slots: local / global request streams
  char *ws = nullptr;
  size_t ws_bytes = 0;
  unsigned char *pin = nullptr;
  size_t pin_bytes = 0;
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned char> gkey;
  int gkernels = 0;
  // tables are identified by a generation number (one per distinct build, 0 = unnamed): the one
  // whose contents ws holds (re-uploaded only when it changes) and the one the graph was
  // captured with (its launch parameters and table pointers depend on them)
  uint64_t ws_gen = 0, graph_gen = 0;
  const void *last_ws = nullptr;
  std::shared_ptr<TableCache> tcache;  // the last tables built on this executor
  // recorded after the last copy into or out of the pinned buffer
  cudaEvent_t pin_ev = nullptr;
  bool pin_ev_live = false;
  // second stream for work independent of the main stream's (a parallel branch of the graph)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// Serving: queued requests and the worker slots that run them.
struct ServeReq {
  int kind = 0, chunk_id = 0;
  std::vector<int> ids;
  bf_solve_params prm{};
  bool done = false;
  bf_status status = BF_OK;
  bf_solve_stats stats{};
  std::chrono::steady_clock::time_point t_submit;
};

struct Server {
  std::mutex qm;
  std::condition_variable qcv, dcv;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, ServeReq> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  int max_batch = 64, max_queue = 1024;
  std::vector<std::unique_ptr<Exec>> slots;
  std::vector<std::thread> workers;
};

struct bf_ctx {
  bf_config cfg{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  size_t bytes = 0;
  Intr intr{};
  // frame store
  int cap = 0;
  float4 *A = nullptr, *B = nullptr;
  unsigned short *C16 = nullptr;  // 16-bit storage: intensity plane (dense verification)
  // TSDF volume (Sec. 5): device arrays, the frames integrated and the pose each used
  bool tsdf_on = false;
  bf_tsdf_config tsdf_cfg{};
  TsdfDev tsdf{};
  std::vector<std::pair<void *, size_t>> tsdf_allocs;
  std::map<int, Pose12> tsdf_integrated;
  int tsdf_call = 0;
  std::map<long long, int> tuned_tile;  // dense decomposition chosen by the autotuner, per frame size/storage
  void *kp_buf = nullptr;         // key-point filter: inputs and results
  size_t kp_cap = 0;
  VerifyPair *vrec = nullptr;     // dense verification: pair records and results
  double *vout = nullptr;
  int vcap = 0;
  float *kx = nullptr, *ky = nullptr;
  std::unordered_map<int, FrameInfo> frames;
  std::vector<int> free_slots;
  int next_slot = 0;
  // staging for host frame uploads
  float *stage = nullptr;
  size_t stage_bytes = 0;
  int *slot_dev = nullptr;
  int slot_dev_cap = 0;
  // correspondence pool
  float4 *cP = nullptr, *cQ = nullptr;
  long long ccap = 0, cused = 0;
  std::unordered_map<uint64_t, std::vector<Seg>> corr;
  std::unordered_map<int, Chunk> chunks;
  // signature of the pair map's layout (an XOR of one hash per segment: pair, position within the
  // pair, pool offset, count; points re-uploaded into the same layout keep it) and a counter bumped
  // whenever a frame id gets a slot; with the problem list and the table parameters they decide
  // whether a solve can reuse the last tables it built
  uint64_t corr_sig = 0, frames_ver = 0, tables_gen = 0;
  // solve executor in use (main, or a serving slot while it holds the context lock)
  Exec main;
  Exec *ex = &main;
  // concurrency: every public call holds mu; serving slots release it while their GPU work runs
  std::mutex mu;
  std::condition_variable busy_cv;  // signalled when in_flight drops
  int in_flight = 0;                // serving batches whose GPU work is running
  cudaEvent_t data_ev = nullptr;    // recorded on the main stream after frame / correspondence uploads
  std::unique_ptr<Server> srv;
  // kernel accounting
  long long launches = 0;
  bool prof = false;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  size_t rec_used = 0;
  // association recording (debug): while on, single-problem solves run kernel by kernel and keep
  // the association of every dense evaluation and the poses it used (the last solve's, on the host)
  bool assoc_rec = false;
  int *rec_dev = nullptr;
  double *rec_pose_dev = nullptr;
  size_t rec_dev_n = 0, rec_pose_n = 0;  // capacities (ints, doubles)
  struct AssocRecord {
    std::vector<int> ids;              // frame ids of the solve, in its local order
    std::vector<int> dp_src, dp_dst;   // directed pairs (local frame indices)
    int n_eval = 0;                    // dense evaluations: n_gn linearisations + the final energy
    std::vector<int> tgt;              // n_eval x n_dp x H x W
    std::vector<double> pose;          // n_eval x n_frames x 12
  } rec_last;
};

// ------------------------------------------------------------------------------- helpers
static bf_status fail(bf_ctx *c, bf_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

static bf_status cuda_fail(bf_ctx *c, cudaError_t e, const char *where) {
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? BF_ERR_OUT_OF_MEMORY : BF_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

static bf_status dalloc(bf_ctx *c, void **p, size_t n, const char *what) {
  *p = nullptr;
  if (n == 0) return BF_OK;
  if (c->cfg.hbm_budget_bytes && c->bytes + n > c->cfg.hbm_budget_bytes)
    return fail(c, BF_ERR_OUT_OF_MEMORY, std::string("HBM budget exceeded allocating ") + what);
  cudaError_t e = cudaMalloc(p, n);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(c, e, what);
  }
  c->bytes += n;
  return BF_OK;
}

static void dfree(bf_ctx *c, void *p, size_t n) {
  if (p) {
    cudaFree(p);
    c->bytes -= n;
  }
}

// Run one launch wrapper (returns the number of kernels it launched) with accounting.
template <typename F>
static void run_k(bf_ctx *c, int kind, F &&f) {
  bf_ctx::Rec *r = nullptr;
  if (c->prof) {
    if (c->rec_used == c->recs.size()) {
      bf_ctx::Rec nr{kind, nullptr, nullptr};
      if (cudaEventCreate(&nr.a) != cudaSuccess || cudaEventCreate(&nr.b) != cudaSuccess) {
        cudaGetLastError();
        c->launches += f();
        return;
      }
      c->recs.push_back(nr);
    }
    r = &c->recs[c->rec_used];
    r->kind = kind;
    cudaEventRecord(r->a, c->ex->st);
  }
  const int n = f();
  c->launches += n;
  if (r) {
    if (n > 0) {
      cudaEventRecord(r->b, c->ex->st);
      ++c->rec_used;
    }
  }
}

static FrameStore frame_store(const bf_ctx *c) {
  FrameStore fs;
  fs.storage = c->cfg.storage;
  fs.W = c->cfg.width;
  fs.H = c->cfg.height;
  const bool f32 = c->cfg.storage == BF_STORE_FP32;
  fs.A = f32 ? c->A : nullptr;
  fs.B = f32 ? c->B : nullptr;
  fs.P16 = f32 ? nullptr : (const uint4 *)c->A;  // 16-bit storage keeps its records in the A buffer
  fs.C16 = f32 ? nullptr : c->C16;
  fs.kx = c->kx;
  fs.ky = c->ky;
  return fs;
}

// grow the frame store to hold at least n slots: FP32 storage keeps two 16-byte planes per
// pixel (A = depth + normal, B = I + grad I), 16-bit storage one 16-byte record plane (in A)
static bf_status ensure_frames(bf_ctx *c, int n) {
  if (n <= c->cap) return BF_OK;
  int ncap = std::max(n, std::max(2 * c->cap, c->cfg.max_frames_hint));
  const size_t HW = (size_t)c->cfg.width * c->cfg.height;
  const bool two = c->cfg.storage == BF_STORE_FP32;
  float4 *nA = nullptr, *nB = nullptr;
  unsigned short *nC = nullptr;
  bf_status s = dalloc(c, (void **)&nA, ncap * HW * sizeof(float4), "frame store");
  if (s) return s;
  s = two ? dalloc(c, (void **)&nB, ncap * HW * sizeof(float4), "frame store")
          : dalloc(c, (void **)&nC, ncap * HW * sizeof(unsigned short), "frame store");
  if (s) {
    dfree(c, nA, ncap * HW * sizeof(float4));
    return s;
  }
  if (c->cap) {
    CK(cudaMemcpyAsync(nA, c->A, c->cap * HW * sizeof(float4), cudaMemcpyDeviceToDevice, c->st), "grow frames");
    if (two)
      CK(cudaMemcpyAsync(nB, c->B, c->cap * HW * sizeof(float4), cudaMemcpyDeviceToDevice, c->st), "grow frames");
    else
      CK(cudaMemcpyAsync(nC, c->C16, c->cap * HW * sizeof(unsigned short), cudaMemcpyDeviceToDevice, c->st),
         "grow frames");
    CK(cudaStreamSynchronize(c->st), "grow frames");
  }
  dfree(c, c->A, c->cap * HW * sizeof(float4));
  if (two) dfree(c, c->B, c->cap * HW * sizeof(float4));
  else dfree(c, c->C16, c->cap * HW * sizeof(unsigned short));
  c->A = nA;
  c->B = nB;
  c->C16 = nC;
  c->cap = ncap;
  return BF_OK;
}

static bf_status ensure_corr(bf_ctx *c, long long n) {
  if (n <= c->ccap) return BF_OK;
  long long ncap = std::max(n, std::max(2 * c->ccap, 1LL << 16));
  if (ncap > 0x7fffffffLL) return fail(c, BF_ERR_INVALID_ARG, "correspondence pool exceeds 2^31 entries");
  float4 *nP = nullptr, *nQ = nullptr;
  bf_status s = dalloc(c, (void **)&nP, ncap * sizeof(float4), "correspondence pool");
  if (s) return s;
  s = dalloc(c, (void **)&nQ, ncap * sizeof(float4), "correspondence pool");
  if (s) {
    dfree(c, nP, ncap * sizeof(float4));
    return s;
  }
  if (c->cused) {
    CK(cudaMemcpyAsync(nP, c->cP, c->cused * sizeof(float4), cudaMemcpyDeviceToDevice, c->st), "grow pool");
    CK(cudaMemcpyAsync(nQ, c->cQ, c->cused * sizeof(float4), cudaMemcpyDeviceToDevice, c->st), "grow pool");
    CK(cudaStreamSynchronize(c->st), "grow pool");
  }
  dfree(c, c->cP, c->ccap * sizeof(float4));
  dfree(c, c->cQ, c->ccap * sizeof(float4));
  c->cP = nP;
  c->cQ = nQ;
  c->ccap = ncap;
  return BF_OK;
}

// ------------------------------------------------------------------------------ config
extern "C" void bf_default_config(bf_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->width = 80;
  cfg->height = 60;
  cfg->fx = cfg->fy = 525.0 * 80.0 / 640.0;
  cfg->cx = (80 - 1) / 2.0;
  cfg->cy = (60 - 1) / 2.0;
  cfg->depth_min = 0.1f;
  cfg->depth_max = 10.0f;
  cfg->storage = BF_STORE_FP32;
  cfg->hbm_budget_bytes = 0;
  cfg->cuda_stream = nullptr;
  cfg->max_frames_hint = 64;
}

extern "C" void bf_default_params(bf_solve_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_gn = 4;
  p->n_pcg = 10;
  p->w_sparse = 1.0;
  p->w_dense = 0.5;
  p->w_photo = 0.1;
  p->w_geo = 1.0;
  p->dense_ramp = 0;
  p->tau_dist = 0.15;
  p->tau_normal = 0.9;
  p->max_angle_deg = 60.0;
  p->precond = BF_PRECOND_BLOCK_JACOBI;
  p->dense_on = 1;
  p->warm_start = 0;
  p->precision = BF_PREC_MIXED;
  p->use_graph = 0;
  p->tile_px = 0;
  p->prune_rmax = 0.0;
  p->prune_rounds = 8;
  p->sparse_mode = BF_SPARSE_BLOCKS;
}

extern "C" const char *bf_status_string(bf_status s) {
  switch (s) {
    case BF_OK: return "ok";
    case BF_ERR_INVALID_ARG: return "invalid argument";
    case BF_ERR_OUT_OF_MEMORY: return "out of memory";
    case BF_ERR_CUDA: return "CUDA error";
    case BF_ERR_NOT_FOUND: return "not found";
    case BF_ERR_SINGULAR: return "singular block";
    case BF_ERR_TIMEOUT: return "timeout";
    case BF_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

extern "C" const char *bf_last_error(bf_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" size_t bf_device_bytes(bf_ctx *ctx) {
  if (!ctx) return 0;
  std::unique_lock<std::mutex> lk(ctx->mu);
  return ctx->bytes;
}

extern "C" bf_status bf_create(const bf_config *cfg, bf_ctx **out) {
  if (!cfg || !out) return BF_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->width < 8 || cfg->height < 8 || cfg->width > 8192 || cfg->height > 8192) return BF_ERR_INVALID_ARG;
  if (!(cfg->fx > 0) || !(cfg->fy > 0)) return BF_ERR_INVALID_ARG;
  if (cfg->storage != BF_STORE_FP32 && cfg->storage != BF_STORE_BF16 && cfg->storage != BF_STORE_FP16)
    return BF_ERR_INVALID_ARG;
  bf_ctx *c = new bf_ctx();
  c->cfg = *cfg;
  if (c->cfg.max_frames_hint <= 0) c->cfg.max_frames_hint = 64;
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return BF_ERR_CUDA;
  }
  if (cfg->cuda_stream) {
    c->st = (cudaStream_t)cfg->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return BF_ERR_CUDA;
    }
    c->own_stream = true;
  }
  c->main.st = c->st;
  if (cudaEventCreateWithFlags(&c->data_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
    return BF_ERR_CUDA;
  }
  c->intr.fx = (float)cfg->fx;
  c->intr.fy = (float)cfg->fy;
  c->intr.cx = (float)cfg->cx;
  c->intr.cy = (float)cfg->cy;
  c->intr.W = cfg->width;
  c->intr.H = cfg->height;
  // kx[x] = fl32((x - cx) / fx), ky[y] = fl32((y - cy) / fy): FP64 then one rounding
  std::vector<float> kx(cfg->width), ky(cfg->height);
  for (int x = 0; x < cfg->width; ++x) kx[x] = (float)(((double)x - cfg->cx) / cfg->fx);
  for (int y = 0; y < cfg->height; ++y) ky[y] = (float)(((double)y - cfg->cy) / cfg->fy);
  bf_status s = dalloc(c, (void **)&c->kx, cfg->width * sizeof(float), "ray tables");
  if (!s) s = dalloc(c, (void **)&c->ky, cfg->height * sizeof(float), "ray tables");
  if (!s) {
    if (cudaMemcpy(c->kx, kx.data(), kx.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->ky, ky.data(), ky.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      s = BF_ERR_CUDA;
    }
  }
  if (s) {
    bf_destroy(c);
    return s;
  }
  *out = c;
  return BF_OK;
}

static void free_exec(bf_ctx *c, Exec &e) {
  if (e.side) cudaStreamDestroy(e.side);
  if (e.ev_fork) cudaEventDestroy(e.ev_fork);
  if (e.ev_join) cudaEventDestroy(e.ev_join);
  e.side = nullptr;
  e.ev_fork = e.ev_join = nullptr;
  if (e.ws) cudaFree(e.ws);
  if (e.gexec) cudaGraphExecDestroy(e.gexec);
  if (e.pin) cudaFreeHost(e.pin);
  if (e.pin_ev) cudaEventDestroy(e.pin_ev);
  e.pin_ev = nullptr;
  e.pin_ev_live = false;
  e.tcache.reset();
  e.ws_gen = e.graph_gen = 0;
  e.last_ws = nullptr;
  c->bytes -= e.ws_bytes;
  e.ws = nullptr;
  e.ws_bytes = 0;
  e.gexec = nullptr;
  e.pin = nullptr;
  e.pin_bytes = 0;
}

extern "C" bf_status bf_serve_stop(bf_ctx *c);

extern "C" bf_status bf_destroy(bf_ctx *c) {
  if (!c) return BF_OK;
  bf_serve_stop(c);
  if (c->st) cudaStreamSynchronize(c->st);
  cudaFree(c->A);
  cudaFree(c->B);
  cudaFree(c->C16);
  for (auto &a : c->tsdf_allocs) cudaFree(a.first);
  cudaFree(c->vrec);
  cudaFree(c->kp_buf);
  cudaFree(c->vout);
  cudaFree(c->kx);
  cudaFree(c->ky);
  cudaFree(c->stage);
  cudaFree(c->slot_dev);
  cudaFree(c->cP);
  cudaFree(c->cQ);
  cudaFree(c->rec_dev);
  cudaFree(c->rec_pose_dev);
  free_exec(c, c->main);
  for (auto &r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (c->data_ev) cudaEventDestroy(c->data_ev);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  cudaGetLastError();
  delete c;
  return BF_OK;
}

// ------------------------------------------------------------------------------- frames
extern "C" bf_status bf_add_frames(bf_ctx *c, int first_id, int n, const float *depth, const float *lum,
                                   int ptr_kind, const double *init_pose) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (n < 0 || (n > 0 && (!depth || !lum)) || (ptr_kind != BF_PTR_HOST && ptr_kind != BF_PTR_DEVICE))
    return fail(c, BF_ERR_INVALID_ARG, "bf_add_frames: bad arguments");
  if (first_id < 0 || (long long)first_id + n > 0x7fffffffLL)
    return fail(c, BF_ERR_INVALID_ARG, "bf_add_frames: bad frame id range");
  if (n == 0) return BF_OK;
  const size_t HW = (size_t)c->cfg.width * c->cfg.height;
  std::vector<int> slots(n);
  int need = c->next_slot;
  bool replaces = false;
  for (int k = 0; k < n; ++k) {
    auto it = c->frames.find(first_id + k);
    if (it == c->frames.end()) ++need;
    else replaces = true;
  }
  // frames read by serving batches in flight must not move or change underneath them
  if (replaces || need > c->cap) c->busy_cv.wait(lk, [&] { return c->in_flight == 0; });
  bf_status s = ensure_frames(c, need);
  if (s) return s;
  for (int k = 0; k < n; ++k) {
    FrameInfo &fi = c->frames[first_id + k];
    if (fi.slot < 0) {
      ++c->frames_ver;
      if (!c->free_slots.empty()) {
        fi.slot = c->free_slots.back();
        c->free_slots.pop_back();
      } else {
        fi.slot = c->next_slot++;
      }
    }
    slots[k] = fi.slot;
    if (init_pose) {
      Pose12 p = from16(init_pose + 16 * k);
      std::memcpy(fi.world, p.data(), sizeof(fi.world));
      fi.has_world = true;
    }
  }
  if (n > c->slot_dev_cap) {
    dfree(c, c->slot_dev, (size_t)c->slot_dev_cap * sizeof(int));
    c->slot_dev = nullptr;
    c->slot_dev_cap = 0;
    s = dalloc(c, (void **)&c->slot_dev, (size_t)std::max(n, 256) * sizeof(int), "slot table");
    if (s) return s;
    c->slot_dev_cap = std::max(n, 256);
  }
  CK(cudaMemcpyAsync(c->slot_dev, slots.data(), n * sizeof(int), cudaMemcpyHostToDevice, c->st), "slots");
  const float *dptr = depth, *lptr = lum;
  if (ptr_kind == BF_PTR_HOST) {
    const size_t need_b = 2 * (size_t)n * HW * sizeof(float);
    if (need_b > c->stage_bytes) {
      dfree(c, c->stage, c->stage_bytes);
      c->stage = nullptr;
      c->stage_bytes = 0;
      s = dalloc(c, (void **)&c->stage, need_b, "frame staging");
      if (s) return s;
      c->stage_bytes = need_b;
    }
    CK(cudaMemcpyAsync(c->stage, depth, n * HW * sizeof(float), cudaMemcpyHostToDevice, c->st), "upload depth");
    CK(cudaMemcpyAsync(c->stage + n * HW, lum, n * HW * sizeof(float), cudaMemcpyHostToDevice, c->st),
       "upload luminance");
    dptr = c->stage;
    lptr = c->stage + n * HW;
  }
  run_k(c, BF_K_PREPROCESS, [&] {
    return launch_preprocess(dptr, lptr, n, c->slot_dev, frame_store(c), c->A, c->B, (uint4 *)c->A, c->C16,
                             c->cfg.depth_min, c->cfg.depth_max, c->st);
  });
  CK(cudaGetLastError(), "preprocess launch");
  CK(cudaEventRecord(c->data_ev, c->st), "data event");
  if (ptr_kind == BF_PTR_HOST) CK(cudaStreamSynchronize(c->st), "preprocess");
  return BF_OK;
}

extern "C" bf_status bf_get_frame_planes(bf_ctx *c, int frame_id, float *out) {
  if (!c || !out) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->frames.find(frame_id);
  if (it == c->frames.end()) return fail(c, BF_ERR_NOT_FOUND, "unknown frame id");
  const size_t HW = (size_t)c->cfg.width * c->cfg.height;
  std::vector<float4> a(HW), b(HW);
  CK(cudaMemcpyAsync(a.data(), c->A + it->second.slot * HW, HW * sizeof(float4), cudaMemcpyDeviceToHost, c->st),
     "planes");
  if (c->cfg.storage == BF_STORE_FP32)
    CK(cudaMemcpyAsync(b.data(), c->B + it->second.slot * HW, HW * sizeof(float4), cudaMemcpyDeviceToHost, c->st),
       "planes");
  CK(cudaStreamSynchronize(c->st), "planes");
  if (c->cfg.storage != BF_STORE_FP32) {
    // unpack the 16-bit records: {D bits, nx | ny, nz | I, Ix | Iy}
    const bool bf = c->cfg.storage == BF_STORE_BF16;
    auto h2f = [bf](uint32_t h) {
      if (bf) {
        const uint32_t u = h << 16;
        float f;
        std::memcpy(&f, &u, 4);
        return f;
      }
      __half_raw r;
      r.x = (unsigned short)h;
      return __half2float(__half(r));
    };
    for (size_t k = 0; k < HW; ++k) {
      uint32_t w[4];
      std::memcpy(w, &a[k], 16);
      float d;
      std::memcpy(&d, &w[0], 4);
      a[k] = make_float4(d, h2f(w[1] & 0xffffu), h2f(w[1] >> 16), h2f(w[2] & 0xffffu));
      b[k] = make_float4(h2f(w[2] >> 16), h2f(w[3] & 0xffffu), h2f(w[3] >> 16), 0.f);
    }
  }
  for (size_t k = 0; k < HW; ++k) {
    out[k] = a[k].x;
    out[HW + k] = a[k].y;
    out[2 * HW + k] = a[k].z;
    out[3 * HW + k] = a[k].w;
    out[4 * HW + k] = b[k].x;
    out[5 * HW + k] = b[k].y;
    out[6 * HW + k] = b[k].z;
  }
  return BF_OK;
}

// ------------------------------------------------------------------ correspondence map
static inline uint64_t mix64(uint64_t x) {  // SplitMix64's finaliser (Steele, Lea, Flood 2014)
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}
static inline uint64_t seg_sig(uint64_t key, size_t pos, const Seg &s) {
  return mix64(key ^ mix64((uint64_t)pos ^ mix64(((uint64_t)(uint32_t)s.off << 32) | (uint32_t)s.cnt)));
}
// Appends a segment to a pair's list, keeping the map's layout signature.
static void corr_push(bf_ctx *c, uint64_t key, const Seg &s) {
  std::vector<Seg> &v = c->corr[key];
  c->corr_sig ^= seg_sig(key, v.size(), s);
  v.push_back(s);
}
// Removes a pair and its segments from the map and the signature.
static void corr_erase(bf_ctx *c, uint64_t key) {
  auto it = c->corr.find(key);
  if (it == c->corr.end()) return;
  for (size_t k = 0; k < it->second.size(); ++k) c->corr_sig ^= seg_sig(key, k, it->second[k]);
  c->corr.erase(it);
}

// ---------------------------------------------------------------------- correspondences
extern "C" bf_status bf_add_correspondences(bf_ctx *c, int frame_i, int frame_j, int n, const float *p_i,
                                            const float *p_j, const float *weight, int ptr_kind) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (n < 0 || frame_i == frame_j || frame_i < 0 || frame_j < 0 || (n > 0 && (!p_i || !p_j)) ||
      (ptr_kind != BF_PTR_HOST && ptr_kind != BF_PTR_DEVICE))
    return fail(c, BF_ERR_INVALID_ARG, "bf_add_correspondences: bad arguments");
  if (n == 0) return BF_OK;
  if (c->cused + n > c->ccap) c->busy_cv.wait(lk, [&] { return c->in_flight == 0; });
  bf_status s = ensure_corr(c, c->cused + n);
  if (s) return s;
  const int swap = frame_i > frame_j ? 1 : 0;
  if (ptr_kind == BF_PTR_HOST) {
    std::vector<float4> P(n), Q(n);
    const float *a = swap ? p_j : p_i;
    const float *b = swap ? p_i : p_j;
    for (int k = 0; k < n; ++k) {
      P[k] = make_float4(a[3 * k], a[3 * k + 1], a[3 * k + 2], weight ? weight[k] : 1.f);
      Q[k] = make_float4(b[3 * k], b[3 * k + 1], b[3 * k + 2], 0.f);
    }
    CK(cudaMemcpyAsync(c->cP + c->cused, P.data(), n * sizeof(float4), cudaMemcpyHostToDevice, c->st), "corr");
    CK(cudaMemcpyAsync(c->cQ + c->cused, Q.data(), n * sizeof(float4), cudaMemcpyHostToDevice, c->st), "corr");
    CK(cudaStreamSynchronize(c->st), "corr");
  } else {
    run_k(c, BF_K_PACK,
          [&] { return launch_pack_corr(p_i, p_j, weight, n, swap, c->cP + c->cused, c->cQ + c->cused, c->st); });
    CK(cudaGetLastError(), "pack corr");
  }
  corr_push(c, pair_key(frame_i, frame_j), Seg{(int)c->cused, n});
  c->cused += n;
  CK(cudaEventRecord(c->data_ev, c->st), "data event");
  return BF_OK;
}

extern "C" bf_status bf_add_correspondences_batch(bf_ctx *c, int n_pairs, const int *pair_ids, const int *offsets,
                                                  const float *p_i, const float *p_j, const float *weight,
                                                  int ptr_kind) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (n_pairs < 0 || (n_pairs > 0 && (!pair_ids || !offsets)) || (ptr_kind != BF_PTR_HOST && ptr_kind != BF_PTR_DEVICE))
    return fail(c, BF_ERR_INVALID_ARG, "bf_add_correspondences_batch: bad arguments");
  if (n_pairs == 0) return BF_OK;
  if (offsets[0] != 0) return fail(c, BF_ERR_INVALID_ARG, "bf_add_correspondences_batch: offsets[0] must be 0");
  for (int k = 0; k < n_pairs; ++k) {
    if (offsets[k + 1] < offsets[k] || pair_ids[2 * k] == pair_ids[2 * k + 1] || pair_ids[2 * k] < 0 ||
        pair_ids[2 * k + 1] < 0)
      return fail(c, BF_ERR_INVALID_ARG, "bf_add_correspondences_batch: bad pair " + std::to_string(k));
  }
  const long long total = offsets[n_pairs];
  if (total == 0) return BF_OK;
  if (!p_i || !p_j) return fail(c, BF_ERR_INVALID_ARG, "bf_add_correspondences_batch: null points");
  if (c->cused + total > c->ccap) c->busy_cv.wait(lk, [&] { return c->in_flight == 0; });
  bf_status s = ensure_corr(c, c->cused + total);
  if (s) return s;
  if (ptr_kind == BF_PTR_HOST) {
    // the caller's arrays go to the device as they are (one copy each, straight from pinned
    // memory when the caller's is pinned) into the upload staging buffer; the packing kernel below
    // then builds the pool records on the device
    const size_t need_b = (size_t)total * (weight ? 7 : 6) * sizeof(float);
    if (need_b > c->stage_bytes) {
      CK(cudaStreamSynchronize(c->st), "staging");
      dfree(c, c->stage, c->stage_bytes);
      c->stage = nullptr;
      c->stage_bytes = 0;
      s = dalloc(c, (void **)&c->stage, need_b, "upload staging");
      if (s) return s;
      c->stage_bytes = need_b;
    }
    float *sp = c->stage, *sq = c->stage + 3 * total, *sw = weight ? c->stage + 6 * total : nullptr;
    CK(cudaMemcpyAsync(sp, p_i, total * 3 * sizeof(float), cudaMemcpyHostToDevice, c->st), "upload p_i");
    CK(cudaMemcpyAsync(sq, p_j, total * 3 * sizeof(float), cudaMemcpyHostToDevice, c->st), "upload p_j");
    if (weight) CK(cudaMemcpyAsync(sw, weight, total * sizeof(float), cudaMemcpyHostToDevice, c->st), "upload w");
    p_i = sp;
    p_j = sq;
    weight = sw;
  }
  {
    // offsets and swap flags to the device (scratch), then one packing kernel
    std::vector<int> meta(2 * (size_t)n_pairs + 1);
    for (int k = 0; k <= n_pairs; ++k) meta[k] = offsets[k];
    for (int k = 0; k < n_pairs; ++k) meta[n_pairs + 1 + k] = pair_ids[2 * k] > pair_ids[2 * k + 1] ? 1 : 0;
    if ((int)meta.size() > c->slot_dev_cap) {
      dfree(c, c->slot_dev, (size_t)c->slot_dev_cap * sizeof(int));
      c->slot_dev = nullptr;
      c->slot_dev_cap = 0;
      s = dalloc(c, (void **)&c->slot_dev, meta.size() * sizeof(int), "scratch table");
      if (s) return s;
      c->slot_dev_cap = (int)meta.size();
    }
    CK(cudaMemcpyAsync(c->slot_dev, meta.data(), meta.size() * sizeof(int), cudaMemcpyHostToDevice, c->st), "meta");
    run_k(c, BF_K_PACK, [&] {
      return launch_pack_corr_batch(p_i, p_j, weight, (int)total, c->slot_dev, c->slot_dev + n_pairs + 1, n_pairs,
                                    c->cP + c->cused, c->cQ + c->cused, c->st);
    });
    CK(cudaGetLastError(), "pack corr");
    CK(cudaStreamSynchronize(c->st), "pack corr");
  }
  for (int k = 0; k < n_pairs; ++k) {
    const int n = offsets[k + 1] - offsets[k];
    if (n == 0) continue;
    corr_push(c, pair_key(pair_ids[2 * k], pair_ids[2 * k + 1]), Seg{(int)(c->cused + offsets[k]), n});
  }
  c->cused += total;
  CK(cudaEventRecord(c->data_ev, c->st), "data event");
  return BF_OK;
}

extern "C" bf_status bf_set_profiling(bf_ctx *c, int enable) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  c->prof = enable != 0;
  return BF_OK;
}

extern "C" bf_status bf_reset_profile(bf_ctx *c) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  c->launches = 0;
  c->rec_used = 0;
  return BF_OK;
}

extern "C" bf_status bf_get_profile(bf_ctx *c, bf_profile *out) {
  if (!c || !out) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  std::memset(out, 0, sizeof(*out));
  CK(cudaStreamSynchronize(c->st), "profile");
  out->launches = c->launches;
  for (size_t k = 0; k < c->rec_used; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->recs[k].a, c->recs[k].b), "profile");
    out->count[c->recs[k].kind] += 1;
    out->ms[c->recs[k].kind] += ms;
  }
  return BF_OK;
}

extern "C" bf_status bf_remove_pair(bf_ctx *c, int frame_i, int frame_j) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->corr.find(pair_key(frame_i, frame_j));
  if (it == c->corr.end()) return fail(c, BF_ERR_NOT_FOUND, "bf_remove_pair: no such pair");
  corr_erase(c, it->first);
  return BF_OK;
}

extern "C" bf_status bf_clear_correspondences(bf_ctx *c) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  c->busy_cv.wait(lk, [&] { return c->in_flight == 0; });  // batches in flight still read the pool
  c->corr.clear();
  c->cused = 0;
  c->corr_sig = 0;
  return BF_OK;
}

// ------------------------------------------------------------------------- solve tables
namespace {

struct Problem {
  std::vector<int> ids;
  std::vector<Pose12> init;
};

struct HostTables {
  int n_frames = 0, n_pairs = 0, n_dp = 0, n_tiles = 0, n_segs = 0, n_vars = 0, n_prob = 0;
  std::vector<int> frame_slot, frame_var, pair_a, pair_b, pair_dp, pair_seg0, pair_seg1;
  std::vector<int> dp_src, dp_dst, dp_pair, dp_dir, dp_tile0, dp_tile1, tile_dp, tile_px0, tile_px1;
  std::vector<int> seg_pair, seg_off, seg_cnt, seg_swap, inc_off, inc, inc_ov, var_frame;
  std::vector<int> prob_var0, prob_var1, prob_pair0, prob_pair1, prob_frame0;
  std::vector<int> prob_tile0, prob_tile1, prob_seg0, prob_seg1;
  int n_wi = 0;                        // target-staged dense work items (0: tiled kernel)
  std::vector<int> wi_off, sw_dp, dp_dst_host;
  std::vector<int> pair_ida, pair_idb;  // frame ids of the pair (for stats)
  std::vector<double> pose;             // n_frames x 12
  long long n_corr = 0;
  std::vector<int> prob_npairs, prob_ndense;
  std::vector<long long> prob_ncorr;
  uint64_t gen = 0;                              // build generation (0: assembled by hand)
  std::shared_ptr<const std::vector<int>> ints;  // the device tables, packed (see pack_ints)
};

// The last tables an executor built, with what they were built from.
struct TableCache {
  std::vector<std::vector<int>> ids;  // frame ids per problem
  uint64_t corr_sig = 0, frames_ver = 0;
  size_t corr_pairs = 0;
  int tile_px = 0, dense_on = 0;
  bool staged = false;
  double max_angle_deg = 0;
  HostTables T;
  uint64_t gen = 0;   // T's generation
  bool lent = false;  // T moved out to a solve in flight (given back by return_tables)
};

constexpr int STAGED_PAIRS_PER_ITEM = 6;

// Build the flattened tables of a set of problems.  force_dense: every pair gets both dense
// directions (debug), else the Sec. 4.3 angle test on the initial poses selects E.
// Sec. 4.3's dense set E: the optical axes (third rotation columns) of the pair's initial poses
// within the maximum angle, tested in FP64.
static inline bool axes_within(const Pose12 &Pa, const Pose12 &Pb, double cos_max) {
  const double dot = (Pa[2] * Pb[2] + Pa[5] * Pb[5]) + Pa[8] * Pb[8];
  return dot > cos_max;
}

// dense work decomposition: explicit tile_px -> tiles of that many pixels; automatic -> the
// target frame staged in shared memory when it fits (one partial per directed pair), else
// 4800-pixel tiles
static void dense_decomposition(const bf_ctx *c, const bf_solve_params &prm, bool &staged, int &tile_px) {
  const int HW = c->cfg.width * c->cfg.height;
  staged = prm.tile_px == 0 && !prm.compensated && !prm.dense_tc &&
           dense_staged_fits(c->cfg.width, c->cfg.height, c->cfg.storage);
  tile_px = prm.tile_px > 0 ? prm.tile_px : (staged ? HW : std::min(HW, 4800));
}

bf_status build_tables_fresh(bf_ctx *c, const std::vector<Problem> &probs, const bf_solve_params &prm,
                             HostTables &T) {
  const int HW = c->cfg.width * c->cfg.height;
  bool staged;
  int tile_px;
  dense_decomposition(c, prm, staged, tile_px);
  T.n_prob = (int)probs.size();
  std::vector<std::vector<std::pair<int, int>>> var_inc;  // per var: (pair, side)
  const double cos_max = std::cos(prm.max_angle_deg * M_PI / 180.0);
  for (int pi = 0; pi < T.n_prob; ++pi) {
    const Problem &P = probs[pi];
    const int n = (int)P.ids.size();
    const int F0 = T.n_frames;
    T.prob_frame0.push_back(F0);
    T.prob_var0.push_back(T.n_vars);
    // frame id -> local index: a direct table when the ids are small, else a hash map
    int id_max = -1;
    bool id_neg = false;
    for (int id : P.ids) {
      id_max = std::max(id_max, id);
      id_neg |= id < 0;
    }
    const bool direct = !id_neg && (long long)id_max <= 8LL * n + 4096;
    std::vector<int> dloc(direct ? id_max + 1 : 0, -1);
    std::unordered_map<int, int> hloc;
    if (!direct) hloc.reserve(n * 2);
    auto local_of = [&](int id) -> int {
      if (direct) return id >= 0 && id <= id_max ? dloc[id] : -1;
      auto it = hloc.find(id);
      return it == hloc.end() ? -1 : it->second;
    };
    for (int k = 0; k < n; ++k) {
      auto it = c->frames.find(P.ids[k]);
      if (it == c->frames.end()) return fail(c, BF_ERR_NOT_FOUND, "solve: unknown frame id " + std::to_string(P.ids[k]));
      if (local_of(P.ids[k]) >= 0)
        return fail(c, BF_ERR_INVALID_ARG, "solve: duplicate frame id " + std::to_string(P.ids[k]));
      if (direct) dloc[P.ids[k]] = k;
      else hloc.emplace(P.ids[k], k);
      T.frame_slot.push_back(it->second.slot);
      if (k == 0) {
        T.frame_var.push_back(-1);
      } else {
        T.frame_var.push_back(T.n_vars);
        T.var_frame.push_back(F0 + k);
        var_inc.emplace_back();
        ++T.n_vars;
      }
      for (int q = 0; q < 12; ++q) T.pose.push_back(P.init[k][q]);
    }
    T.n_frames += n;
    T.prob_var1.push_back(T.n_vars);
    // pairs with correspondences among the problem's frames, in (a, b) order, each with its
    // segment list (one map lookup per pair)
    struct PEnt {
      int a, b;
      const std::vector<Seg> *segs;
    };
    std::vector<PEnt> plist;
    if ((long long)n * (n - 1) / 2 <= (long long)c->corr.size()) {
      for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
          auto it = c->corr.find(pair_key(P.ids[a], P.ids[b]));
          if (it != c->corr.end()) plist.push_back({a, b, &it->second});
        }
    } else {
      plist.reserve(c->corr.size());
      for (auto &kv : c->corr) {
        const int la = local_of((int)(kv.first >> 32)), lb = local_of((int)(kv.first & 0xffffffffu));
        if (la < 0 || lb < 0) continue;
        plist.push_back({std::min(la, lb), std::max(la, lb), &kv.second});
      }
      std::sort(plist.begin(), plist.end(),
                [](const PEnt &x, const PEnt &y) { return x.a != y.a ? x.a < y.a : x.b < y.b; });
    }
    T.prob_pair0.push_back(T.n_pairs);
    T.prob_tile0.push_back(T.n_tiles);
    T.prob_seg0.push_back(T.n_segs);
    int ndense = 0;
    long long ncorr = 0;
    for (const PEnt &ab : plist) {
      const int a = ab.a, b = ab.b;
      const int p = T.n_pairs++;
      T.pair_a.push_back(F0 + a);
      T.pair_b.push_back(F0 + b);
      T.pair_ida.push_back(P.ids[a]);
      T.pair_idb.push_back(P.ids[b]);
      const std::vector<Seg> &segs = *ab.segs;
      long long pair_n = 0;
      for (const Seg &sg : segs) pair_n += sg.cnt;
      if (pair_n < 3)  // fewer than 3 matches determine no rigid transform (Sec. 4.1.1)
        return fail(c, BF_ERR_INVALID_ARG, "a frame pair of the solve has fewer than 3 correspondences");
      T.pair_seg0.push_back(T.n_segs);
      const int swap = P.ids[a] > P.ids[b] ? 1 : 0;  // pool stores the smaller id's point first
      for (const Seg &sg : segs) {
        T.seg_pair.push_back(p);
        T.seg_off.push_back(sg.off);
        T.seg_cnt.push_back(sg.cnt);
        T.seg_swap.push_back(swap);
        ncorr += sg.cnt;
        ++T.n_segs;
      }
      T.pair_seg1.push_back(T.n_segs);
      // dense set E: optical axes within max_angle at the initial poses (FP64)
      const bool dense = prm.dense_on && axes_within(P.init[a], P.init[b], cos_max);
      for (int dir = 0; dir < 2; ++dir) {
        if (!dense) {
          T.pair_dp.push_back(-1);
          continue;
        }
        const int d = T.n_dp++;
        T.pair_dp.push_back(d);
        T.dp_src.push_back(dir == 0 ? F0 + a : F0 + b);
        T.dp_dst.push_back(dir == 0 ? F0 + b : F0 + a);
        T.dp_pair.push_back(p);
        T.dp_dir.push_back(dir);
        T.dp_tile0.push_back(T.n_tiles);
        for (int px = 0; px < HW; px += tile_px) {
          T.tile_dp.push_back(d);
          T.tile_px0.push_back(px);
          T.tile_px1.push_back(std::min(HW, px + tile_px));
          ++T.n_tiles;
        }
        T.dp_tile1.push_back(T.n_tiles);
        if (staged) T.dp_dst_host.push_back(dir == 0 ? F0 + b : F0 + a);
      }
      if (dense) ++ndense;
      if (a != 0) var_inc[T.frame_var[F0 + a]].push_back({p, 0});
      if (b != 0) var_inc[T.frame_var[F0 + b]].push_back({p, 1});
    }
    T.prob_pair1.push_back(T.n_pairs);
    T.prob_tile1.push_back(T.n_tiles);
    T.prob_seg1.push_back(T.n_segs);
    T.prob_npairs.push_back((int)plist.size());
    T.prob_ndense.push_back(ndense);
    T.prob_ncorr.push_back(ncorr);
    T.n_corr += ncorr;
  }
  if (staged && T.n_dp > 0) {
    // group the directed pairs by target frame, at most STAGED_PAIRS_PER_ITEM per work item (one per
    // warp quad: many small items keep the one-CTA-per-SM grid balanced)
    // (a stable counting sort by target frame)
    std::vector<int> order(T.n_dp), start(T.n_frames + 1, 0);
    for (int d = 0; d < T.n_dp; ++d) ++start[T.dp_dst_host[d] + 1];
    for (int f = 0; f < T.n_frames; ++f) start[f + 1] += start[f];
    for (int d = 0; d < T.n_dp; ++d) order[start[T.dp_dst_host[d]]++] = d;
    // a target with n directed pairs gets ceil(n / 6) items of near-equal size (15 pairs: 5, 5, 5
    // rather than 6, 6, 3), and the items are launched largest first, so the launch's last wave
    // holds the short items (one CTA per SM: the tail is one item long)
    std::vector<std::array<int, 2>> items;  // (first index into order, size)
    for (int k = 0; k < T.n_dp;) {
      int e = k;
      while (e < T.n_dp && T.dp_dst_host[order[e]] == T.dp_dst_host[order[k]]) ++e;
      const int n = e - k, m = (n + STAGED_PAIRS_PER_ITEM - 1) / STAGED_PAIRS_PER_ITEM;
      for (int q = 0, at = k; q < m; ++q) {
        const int sz = n / m + (q < n % m ? 1 : 0);
        items.push_back({at, sz});
        at += sz;
      }
      k = e;
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::array<int, 2> &x, const std::array<int, 2> &y) { return x[1] > y[1]; });
    T.wi_off.push_back(0);
    for (const auto &it : items) {
      for (int q = 0; q < it[1]; ++q) T.sw_dp.push_back(order[it[0] + q]);
      T.wi_off.push_back((int)T.sw_dp.size());
    }
    T.n_wi = (int)items.size();
  } else {
    T.wi_off.push_back(0);
  }
  T.inc_off.assign(T.n_vars + 1, 0);
  for (int v = 0; v < T.n_vars; ++v) T.inc_off[v + 1] = T.inc_off[v] + (int)var_inc[v].size();
  for (int v = 0; v < T.n_vars; ++v)
    for (auto &e : var_inc[v]) {
      T.inc.push_back(2 * e.first + e.second);
      const int other = e.second == 0 ? T.pair_b[e.first] : T.pair_a[e.first];
      T.inc_ov.push_back(T.frame_var[other]);
    }
  return BF_OK;
}

// Device arena: bump allocations aligned to 256 bytes.
struct Arena {
  char *base;
  size_t off = 0;
  template <typename X>
  X *take(size_t n) {
    X *p = (X *)(base + off);
    off += (n * sizeof(X) + 255) & ~(size_t)255;
    return p;
  }
};

struct DevSolve {
  Tables t;
  double *pose;
  float *pairM;  // [n_pairs][2][12] pair transforms at the current poses
  void *dpart, *spart;
  float *srmax;
  int *srarg;
  void *pairblk, *pairen;
  float *pairoff;
  void *Dd, *rhs;
  float *Df, *Minv;
  int *vflags, *pflags;
  float *x, *r, *z, *p, *q, *p1;
  double *energy;  // (n_gn + 1) x n_prob x 4
  int *assoc;
  // matrix-free sparse term: dense-only pair blocks / diagonal blocks and the per-pair products
  void *pairblk2, *pairen2, *Dd2, *rhs2;
  float *Minv2, *mfy;
  int *vflags2;
  bool matfree;
  // persistent batched solve: its work queue (batch_queue_bytes) and item count
  void *bq;
  long long bq_total;
  bool persistent;
  void *coop;      // cooperative PCG state (barrier, error flag, partials)
  int *derr;       // set by the staged dense kernel if its bulk copies did not land
  int coop_grid;   // > 0: one large problem solved by the cooperative PCG
  int cluster;     // > 0: one large problem solved on a thread-block cluster of this many CTAs
  // association recording (debug, bf_debug_record_association): per dense evaluation e, the
  // targets of every directed pair (n_dp x H x W ints from rec + e n_dp H W) and the poses it
  // was evaluated at (n_frames x 12 doubles from rec_pose + e n_frames 12); nullptr when off
  int *rec = nullptr;
  double *rec_pose = nullptr;
};

// The cooperative multi-CTA PCG serves single-problem solves with at least this many free frames.
constexpr int COOP_MIN_VARS = 32;

// Cluster PCG (vectors replicated in shared memory) while the replicas fit.
constexpr size_t CLUSTER_SMEM_MAX = 200 * 1024;

int cluster_for(const HostTables &T, int variant, bool matfree) {
  if (T.n_prob != 1 || T.n_vars == 0 || matfree) return 0;
  if (variant == BF_PCG_CTA || variant == BF_PCG_GRID) return 0;
  if (variant == BF_PCG_AUTO && T.n_vars < COOP_MIN_VARS) return 0;
  const int cl = cluster_size_max();
  if (cluster_smem_bytes(T.n_vars, cl) > CLUSTER_SMEM_MAX) return 0;
  // automatic choice: the cluster only while its CTAs keep the blocks in shared memory (300
  // keyframes: 103 us per 20-iteration solve against 265 us for the grid-cooperative kernel;
  // 2000 keyframes, blocks in global memory: 982 us against 593 us for 30 iterations)
  if (variant == BF_PCG_AUTO && !cluster_cache_fits(T.n_vars, cl, T.inc_off.data())) return 0;
  return cl;
}

// The matrix-free sparse term is offered by the grid-cooperative and per-problem kernels only.
int coop_grid_for(const HostTables &T, int variant, bool matfree) {
  if (T.n_prob != 1 || T.n_vars == 0 || variant == BF_PCG_CTA) return 0;
  if (variant == BF_PCG_GRID) return coop_grid_size(T.n_vars);
  if (variant == BF_PCG_AUTO && T.n_vars < COOP_MIN_VARS) return 0;
  return cluster_for(T, variant, matfree) == 0 ? coop_grid_size(T.n_vars) : 0;
}

// The persistent batched solve serves tiled dense work, the per-problem PCG kernel and assembled
// sparse blocks.
bool persistent_for(const HostTables &T, int variant, bool matfree) {
  return T.n_wi == 0 && !matfree && cluster_for(T, variant, matfree) == 0 && coop_grid_for(T, variant, matfree) == 0;
}

long long batch_items(const HostTables &T, int n_gn) {
  std::vector<int> L(T.n_prob);
  for (int p = 0; p < T.n_prob; ++p)
    L[p] = (T.prob_tile1[p] - T.prob_tile0[p]) + (T.prob_seg1[p] - T.prob_seg0[p]);
  return batch_total_items(L.data(), T.n_prob, n_gn);
}

size_t layout(const HostTables &T, int n_gn, int n_int, char *base, DevSolve *D, size_t acc_size, int HW,
              bool want_assoc, int variant, bool matfree, bool persistent) {
  Arena a{base};
  int *ib = a.take<int>(n_int);
  double *pose = a.take<double>(T.n_frames * 12);
  float *pairM = a.take<float>((size_t)T.n_pairs * 24);
  char *dpart = a.take<char>((size_t)T.n_tiles * NPD * acc_size);
  char *spart = a.take<char>((size_t)T.n_segs * NPART * acc_size);
  float *srmax = a.take<float>(T.n_segs);
  int *srarg = a.take<int>(T.n_segs);
  char *pairblk = a.take<char>((size_t)T.n_pairs * PAIRBLK * acc_size);
  char *pairen = a.take<char>((size_t)T.n_pairs * PAIREN * acc_size);
  float *pairoff = a.take<float>((size_t)T.n_pairs * 36);
  char *Dd = a.take<char>((size_t)T.n_vars * 36 * acc_size);
  char *rhs = a.take<char>((size_t)T.n_vars * 6 * acc_size);
  float *Df = a.take<float>((size_t)T.n_vars * 36);
  float *Minv = a.take<float>((size_t)T.n_vars * 36);
  int *vflags = a.take<int>(T.n_vars);
  int *pflags = a.take<int>(T.n_prob);
  float *x = a.take<float>((size_t)T.n_vars * 6);
  float *r = a.take<float>((size_t)T.n_vars * 6);
  float *z = a.take<float>((size_t)T.n_vars * 6);
  float *p = a.take<float>((size_t)T.n_vars * 6);
  float *q = a.take<float>((size_t)T.n_vars * 6);
  float *p1 = a.take<float>((size_t)T.n_vars * 6);
  const size_t nm = matfree ? 1 : 0;
  char *pairblk2 = a.take<char>(nm * T.n_pairs * PAIRBLK * acc_size);
  char *pairen2 = a.take<char>(nm * T.n_pairs * PAIREN * acc_size);
  char *Dd2 = a.take<char>(nm * T.n_vars * 36 * acc_size);
  char *rhs2 = a.take<char>(nm * T.n_vars * 6 * acc_size);
  float *Minv2 = a.take<float>(nm * T.n_vars * 36);
  float *mfy = a.take<float>(nm * T.n_pairs * 12);
  int *vflags2 = a.take<int>(nm * T.n_vars);
  const int cg = coop_grid_for(T, variant, matfree);
  void *coop = a.take<char>(cg > 0 ? coop_mem_bytes(cg) : 256);
  const bool pers = persistent && persistent_for(T, variant, matfree);
  const long long bq_total = pers ? batch_items(T, n_gn) : 0;
  void *bq = a.take<char>(pers ? batch_queue_bytes(T.n_prob, bq_total) : 0);
  double *energy = a.take<double>((size_t)(n_gn + 1) * T.n_prob * PAIREN);
  int *derr = a.take<int>(1);
  int *assoc = want_assoc ? a.take<int>(HW) : nullptr;
  if (D) {
    D->pose = pose;
    D->pairM = pairM;
    D->dpart = dpart;
    D->spart = spart;
    D->srmax = srmax;
    D->srarg = srarg;
    D->pairblk = pairblk;
    D->pairen = pairen;
    D->pairoff = pairoff;
    D->Dd = Dd;
    D->rhs = rhs;
    D->Df = Df;
    D->Minv = Minv;
    D->vflags = vflags;
    D->pflags = pflags;
    D->x = x;
    D->r = r;
    D->z = z;
    D->p = p;
    D->q = q;
    D->p1 = p1;
    D->pairblk2 = pairblk2;
    D->pairen2 = pairen2;
    D->Dd2 = Dd2;
    D->rhs2 = rhs2;
    D->Minv2 = Minv2;
    D->mfy = mfy;
    D->vflags2 = vflags2;
    D->matfree = matfree;
    D->bq = bq;
    D->bq_total = bq_total;
    D->persistent = pers;
    D->coop = coop;
    D->coop_grid = cg;
    D->cluster = cluster_for(T, variant, matfree);
    D->energy = energy;
    D->derr = derr;
    D->assoc = assoc;
    // table pointers into ib, in the order of pack_ints
    int *w = ib;
    auto nxt = [&](size_t n) {
      int *r_ = w;
      w += n;
      return r_;
    };
    Tables &t = D->t;
    t.n_frames = T.n_frames;
    t.n_pairs = T.n_pairs;
    t.n_dp = T.n_dp;
    t.n_tiles = T.n_tiles;
    t.n_segs = T.n_segs;
    t.n_vars = T.n_vars;
    t.n_prob = T.n_prob;
    t.frame_slot = nxt(T.frame_slot.size());
    t.frame_var = nxt(T.frame_var.size());
    t.pair_a = nxt(T.pair_a.size());
    t.pair_b = nxt(T.pair_b.size());
    t.pair_dp = nxt(T.pair_dp.size());
    t.pair_seg0 = nxt(T.pair_seg0.size());
    t.pair_seg1 = nxt(T.pair_seg1.size());
    t.dp_src = nxt(T.dp_src.size());
    t.dp_dst = nxt(T.dp_dst.size());
    t.dp_pair = nxt(T.dp_pair.size());
    t.dp_dir = nxt(T.dp_dir.size());
    t.dp_tile0 = nxt(T.dp_tile0.size());
    t.dp_tile1 = nxt(T.dp_tile1.size());
    t.tile_dp = nxt(T.tile_dp.size());
    t.tile_px0 = nxt(T.tile_px0.size());
    t.tile_px1 = nxt(T.tile_px1.size());
    t.seg_pair = nxt(T.seg_pair.size());
    t.seg_off = nxt(T.seg_off.size());
    t.seg_cnt = nxt(T.seg_cnt.size());
    t.seg_swap = nxt(T.seg_swap.size());
    t.inc_off = nxt(T.inc_off.size());
    t.inc = nxt(T.inc.size());
    t.inc_ov = nxt(T.inc_ov.size());
    t.var_frame = nxt(T.var_frame.size());
    t.prob_var0 = nxt(T.prob_var0.size());
    t.prob_var1 = nxt(T.prob_var1.size());
    t.prob_pair0 = nxt(T.prob_pair0.size());
    t.prob_pair1 = nxt(T.prob_pair1.size());
    t.prob_tile0 = nxt(T.prob_tile0.size());
    t.prob_tile1 = nxt(T.prob_tile1.size());
    t.prob_seg0 = nxt(T.prob_seg0.size());
    t.prob_seg1 = nxt(T.prob_seg1.size());
    t.n_wi = T.n_wi;
    t.wi_off = nxt(T.wi_off.size());
    t.sw_dp = nxt(T.sw_dp.size());
  }
  return a.off;
}

std::vector<int> pack_ints(const HostTables &T) {
  std::vector<int> v;
  for (const std::vector<int> *x :
       {&T.frame_slot, &T.frame_var, &T.pair_a, &T.pair_b, &T.pair_dp, &T.pair_seg0, &T.pair_seg1, &T.dp_src,
        &T.dp_dst, &T.dp_pair, &T.dp_dir, &T.dp_tile0, &T.dp_tile1, &T.tile_dp, &T.tile_px0, &T.tile_px1,
        &T.seg_pair, &T.seg_off, &T.seg_cnt, &T.seg_swap, &T.inc_off, &T.inc, &T.inc_ov, &T.var_frame, &T.prob_var0,
        &T.prob_var1, &T.prob_pair0, &T.prob_pair1, &T.prob_tile0, &T.prob_tile1, &T.prob_seg0, &T.prob_seg1,
        &T.wi_off, &T.sw_dp})
    v.insert(v.end(), x->begin(), x->end());
  return v;
}

// Tables of a set of problems.  The executor keeps the last tables it built: a solve over the
// same problems with the same pairs, frame slots, dense decomposition and dense set (the angle
// test at the new initial poses gives the same E) takes a copy of them with the new initial
// poses instead of rebuilding them (the steady state of repeated global solves).
bf_status build_tables(bf_ctx *c, const std::vector<Problem> &probs, const bf_solve_params &prm, HostTables &T) {
  bool staged;
  int tile_px;
  dense_decomposition(c, prm, staged, tile_px);
  const double cos_max = std::cos(prm.max_angle_deg * M_PI / 180.0);
  Exec &ex = *c->ex;
  if (ex.tcache) {
    TableCache &tc = *ex.tcache;
    bool hit = !tc.lent && tc.corr_sig == c->corr_sig && tc.corr_pairs == c->corr.size() && tc.frames_ver == c->frames_ver &&
               tc.tile_px == tile_px &&
               tc.staged == staged && tc.dense_on == prm.dense_on && tc.max_angle_deg == prm.max_angle_deg &&
               tc.ids.size() == probs.size();
    for (size_t q = 0; hit && q < probs.size(); ++q) hit = tc.ids[q] == probs[q].ids;
    const HostTables &C = tc.T;
    for (int q = 0; hit && q < C.n_prob; ++q) {
      const int F0 = C.prob_frame0[q];
      const Problem &P = probs[q];
      for (int p = C.prob_pair0[q]; hit && p < C.prob_pair1[q]; ++p) {
        const bool dense =
            prm.dense_on && axes_within(P.init[C.pair_a[p] - F0], P.init[C.pair_b[p] - F0], cos_max);
        hit = dense == (C.pair_dp[2 * p] >= 0);
      }
    }
    if (hit) {
      // lent to this solve instead of copied (about 0.4 MB of tables for 300 keyframes); the
      // solve gives them back when it finishes
      T = std::move(tc.T);
      tc.lent = true;
      T.pose.clear();
      for (const Problem &P : probs)
        for (const Pose12 &x : P.init) T.pose.insert(T.pose.end(), x.begin(), x.end());
      return BF_OK;
    }
  }
  ex.tcache.reset();
  T = HostTables{};
  bf_status s = build_tables_fresh(c, probs, prm, T);
  if (s) return s;
  T.ints = std::make_shared<const std::vector<int>>(pack_ints(T));
  T.gen = ++c->tables_gen;
  auto tc = std::make_shared<TableCache>();
  tc->ids.reserve(probs.size());
  for (const Problem &P : probs) tc->ids.push_back(P.ids);
  tc->corr_sig = c->corr_sig;
  tc->corr_pairs = c->corr.size();
  tc->frames_ver = c->frames_ver;
  tc->tile_px = tile_px;
  tc->staged = staged;
  tc->dense_on = prm.dense_on;
  tc->max_angle_deg = prm.max_angle_deg;
  tc->T = T;
  tc->gen = T.gen;
  ex.tcache = std::move(tc);
  return BF_OK;
}

// Marks the end of the copies queued so far into or out of the executor's pinned buffer.
bf_status pin_used(bf_ctx *c) {
  Exec &e = *c->ex;
  if (!e.pin_ev) CK(cudaEventCreateWithFlags(&e.pin_ev, cudaEventDisableTiming), "pinned staging event");
  CK(cudaEventRecord(e.pin_ev, e.st), "pinned staging event");
  e.pin_ev_live = true;
  return BF_OK;
}

bf_status ensure_pinned(bf_ctx *c, size_t n) {
  if (n <= c->ex->pin_bytes) return BF_OK;
  CK(cudaStreamSynchronize(c->ex->st), "pinned staging");
  if (c->ex->pin) cudaFreeHost(c->ex->pin);
  c->ex->pin = nullptr;
  c->ex->pin_bytes = 0;
  const size_t nb = std::max(n, (size_t)1 << 16);
  CK(cudaMallocHost((void **)&c->ex->pin, nb), "pinned staging");
  c->ex->pin_bytes = nb;
  return BF_OK;
}

bf_status prepare(bf_ctx *c, const HostTables &T, int n_gn, size_t acc_size, bool want_assoc, DevSolve &D,
                  int variant = BF_PCG_AUTO, bool matfree = false, bool persistent = false) {
  std::shared_ptr<const std::vector<int>> ints_p = T.ints;
  if (!ints_p) ints_p = std::make_shared<const std::vector<int>>(pack_ints(T));
  const std::vector<int> &ints = *ints_p;
  const int HW = c->cfg.width * c->cfg.height;
  const size_t need =
      layout(T, n_gn, ints.size(), nullptr, nullptr, acc_size, HW, want_assoc, variant, matfree, persistent) + 256;
  if (need > c->ex->ws_bytes) {
    const size_t nb = std::max(need, c->ex->ws_bytes * 3 / 2);
    CK(cudaStreamSynchronize(c->ex->st), "workspace");
    dfree(c, c->ex->ws, c->ex->ws_bytes);
    c->ex->ws = nullptr;
    c->ex->ws_bytes = 0;
    // the new allocation may come back at the old address with other contents: forget what the
    // old workspace held so the tables are uploaded again
    c->ex->last_ws = nullptr;
    c->ex->ws_gen = 0;
    bf_status s = dalloc(c, (void **)&c->ex->ws, nb, "solve workspace");
    if (s) return s;
    c->ex->ws_bytes = nb;
  }
  layout(T, n_gn, ints.size(), c->ex->ws, &D, acc_size, HW, want_assoc, variant, matfree, persistent);
  const bool same_tables = c->ex->last_ws == (const void *)c->ex->ws && T.gen != 0 && c->ex->ws_gen == T.gen;
  if (!ints.empty() && !same_tables) {
    CK(cudaMemcpyAsync((void *)D.t.frame_slot, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, c->ex->st),
       "upload tables");
    CK(cudaStreamSynchronize(c->ex->st), "upload tables");
    c->ex->ws_gen = T.gen;
    c->ex->last_ws = c->ex->ws;
  }
  bf_status s = ensure_pinned(c, T.pose.size() * sizeof(double));
  if (s) return s;
  // the pinned buffer may still feed or receive the previous solve's copies: wait for those
  // alone, not for the kernels queued since (frame preprocessing runs on while the host prepares)
  if (c->ex->pin_ev_live) CK(cudaEventSynchronize(c->ex->pin_ev), "pinned staging");
  std::memcpy(c->ex->pin, T.pose.data(), T.pose.size() * sizeof(double));
  CK(cudaMemcpyAsync(D.pose, c->ex->pin, T.pose.size() * sizeof(double), cudaMemcpyHostToDevice, c->ex->st),
     "upload poses");
  s = pin_used(c);
  if (s) return s;
  if (T.n_prob) CK(cudaMemsetAsync(D.pflags, 0, T.n_prob * sizeof(int), c->ex->st), "pflags");
  CK(cudaMemsetAsync(D.derr, 0, sizeof(int), c->ex->st), "dense status");
  return BF_OK;
}

// The executor's second stream (created on first use), or nullptr when kernels are timed one
// by one (profiling) or it cannot be created: the caller then stays on the main stream.
static cudaStream_t side_stream(bf_ctx *c) {
  Exec &e = *c->ex;
  if (c->prof) return nullptr;
  if (!e.side) {
    if (cudaStreamCreateWithFlags(&e.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e.ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (e.side) cudaStreamDestroy(e.side);
      if (e.ev_fork) cudaEventDestroy(e.ev_fork);
      e.side = nullptr;
      e.ev_fork = e.ev_join = nullptr;
      return nullptr;
    }
  }
  return e.side;
}

// One Gauss-Newton iteration's linearisation at the pair transforms in D.pairM: dense + sparse
// partials, merge.  The sparse kernel does not depend on the dense one: it runs on the second
// stream (a parallel branch of the captured graph), where it fills the SMs the dense launch's
// last wave leaves idle, and the merge waits for both.
template <typename Acc>
void linearise(bf_ctx *c, DevSolve &D, const bf_solve_params &prm, double wd, int mode, int *rec = nullptr) {
  const Tables &t = D.t;
  cudaStream_t side = t.n_segs > 0 ? side_stream(c) : nullptr;
  if (side) {
    cudaEventRecord(c->ex->ev_fork, c->ex->st);
    cudaStreamWaitEvent(side, c->ex->ev_fork, 0);
  }
  Gates g;
  g.tau_d2 = (float)(prm.tau_dist * prm.tau_dist);
  g.tau_n = (float)prm.tau_normal;
  run_k(c, BF_K_DENSE, [&] {
    if (t.n_wi > 0)
      return launch_dense_staged<Acc>(mode, t, frame_store(c), c->intr, D.pairM, g, (float)(wd * prm.w_geo),
                                      (float)(wd * prm.w_photo), (Acc *)D.dpart, D.derr, rec, c->ex->st);
    if (prm.dense_tc && mode == MODE_ACCUM && !rec)
      return launch_dense_tc<Acc>(t, frame_store(c), c->intr, D.pairM, g, (float)(wd * prm.w_geo),
                                  (float)(wd * prm.w_photo), (Acc *)D.dpart, D.derr, prm.dense_tc, c->ex->st);
    return launch_dense<Acc>(mode, t, frame_store(c), c->intr, D.pairM, g, (float)(wd * prm.w_geo),
                             (float)(wd * prm.w_photo), (Acc *)D.dpart, rec, c->ex->st, prm.compensated != 0);
  });
  run_k(c, BF_K_SPARSE, [&] {
    return launch_sparse<Acc>(mode, t, c->cP, c->cQ, D.pairM, (float)prm.w_sparse, (Acc *)D.spart, D.srmax,
                              D.srarg, side ? side : c->ex->st);
  });
  if (side) {
    cudaEventRecord(c->ex->ev_join, side);
    cudaStreamWaitEvent(c->ex->st, c->ex->ev_join, 0);
  }
  run_k(c, BF_K_MERGE, [&] {
    if (mode == MODE_ENERGY)  // the energy record alone
      return launch_pair_energy<Acc>(t, (const Acc *)D.dpart, (const Acc *)D.spart, (Acc *)D.pairen, c->ex->st);
    return launch_pair_merge<Acc, Acc>(t, D.pose, (const Acc *)D.dpart, (const Acc *)D.spart, (Acc *)D.pairblk,
                                       (Acc *)D.pairen, D.pairoff, c->ex->st);
  });
}

double wdense_at(const bf_solve_params &prm, int k) {
  return prm.dense_ramp ? prm.w_dense * (k + 1) / prm.n_gn : prm.w_dense;
}

// The whole Gauss-Newton loop as one persistent launch (batch.cu): same weights, gates and
// buffers as the launch sequence below.
template <typename Acc>
bf_status run_gn_batch(bf_ctx *c, const bf_solve_params &prm, DevSolve &D) {
  BatchArgs a;
  a.t = D.t;
  a.fs = frame_store(c);
  a.in = c->intr;
  a.gates.tau_d2 = (float)(prm.tau_dist * prm.tau_dist);
  a.gates.tau_n = (float)prm.tau_normal;
  a.P = c->cP;
  a.Q = c->cQ;
  a.w_sparse = (float)prm.w_sparse;
  for (int k = 0; k <= prm.n_gn; ++k) {
    // iteration k's dense weight; the final energy uses the last iteration's
    const double wd = k < prm.n_gn ? wdense_at(prm, k) : (prm.n_gn > 0 ? wdense_at(prm, prm.n_gn - 1) : prm.w_dense);
    a.wg[k] = (float)(wd * prm.w_geo);
    a.wp[k] = (float)(wd * prm.w_photo);
  }
  a.n_gn = prm.n_gn;
  a.n_pcg = prm.n_pcg;
  a.precond = prm.precond;
  a.pose = D.pose;
  a.pairM = D.pairM;
  a.dpart = D.dpart;
  a.spart = D.spart;
  a.srmax = D.srmax;
  a.srarg = D.srarg;
  a.pairblk = D.pairblk;
  a.pairen = D.pairen;
  a.pairoff = D.pairoff;
  a.Dd = D.Dd;
  a.rhs = D.rhs;
  a.Df = D.Df;
  a.Minv = D.Minv;
  a.vflags = D.vflags;
  a.pflags = D.pflags;
  a.x = D.x;
  a.r = D.r;
  a.z = D.z;
  a.p = D.p;
  a.q = D.q;
  a.energy = D.energy;
  int rc = 0;
  run_k(c, BF_K_BATCH, [&] {
    rc = launch_batch<Acc>(a, D.bq, D.bq_total, c->ex->st);
    return rc < 0 ? 0 : rc;
  });
  if (rc < 0) return cuda_fail(c, cudaGetLastError(), "persistent batch launch");
  CK(cudaGetLastError(), "persistent batch");
  return BF_OK;
}

template <typename Acc>
bf_status run_gn(bf_ctx *c, const HostTables &T, const bf_solve_params &prm, DevSolve &D) {
  if (D.persistent) return run_gn_batch<Acc>(c, prm, D);
  const Tables &t = D.t;
  run_k(c, BF_K_XFORM, [&] { return launch_pair_xform(t, D.pose, D.pairM, c->ex->st); });
  const size_t rec_n = (size_t)T.n_dp * c->cfg.width * c->cfg.height;
  auto record_poses = [&](int e) {
    if (D.rec_pose)
      cudaMemcpyAsync(D.rec_pose + (size_t)e * T.n_frames * 12, D.pose, (size_t)T.n_frames * 12 * sizeof(double),
                      cudaMemcpyDeviceToDevice, c->ex->st);
  };
  for (int k = 0; k < prm.n_gn; ++k) {
    const double wd = wdense_at(prm, k);
    record_poses(k);
    linearise<Acc>(c, D, prm, wd, MODE_ACCUM, D.rec ? D.rec + (size_t)k * rec_n : nullptr);
    run_k(c, BF_K_ASSEMBLE, [&] {
      return launch_assemble<Acc>(t, (const Acc *)D.pairblk, prm.precond, (Acc *)D.Dd, (Acc *)D.rhs, D.Df, D.Minv,
                                  D.vflags, c->ex->st);
    });
    MatFree mf{};
    if (D.matfree) {
      // the matvec's blocks hold the dense term alone: merge and assemble again without the
      // sparse segments (pair blocks, off-diagonal FP32 copies and diagonal blocks; the
      // preconditioner and right-hand side above keep the sparse term)
      run_k(c, BF_K_MERGE, [&] {
        return launch_pair_merge<Acc, Acc>(t, D.pose, (const Acc *)D.dpart, (const Acc *)nullptr,
                                           (Acc *)D.pairblk2, (Acc *)D.pairen2, D.pairoff, c->ex->st);
      });
      run_k(c, BF_K_ASSEMBLE, [&] {
        return launch_assemble<Acc>(t, (const Acc *)D.pairblk2, prm.precond, (Acc *)D.Dd2, (Acc *)D.rhs2, D.Df,
                                    D.Minv2, D.vflags2, c->ex->st);
      });
      mf.P = c->cP;
      mf.Q = c->cQ;
      mf.pose = D.pose;
      mf.w_sparse = (float)prm.w_sparse;
      mf.mfy = D.mfy;
    }
    // the PCG kernel also records this linearisation's energy and applies the pose update; the
    // per-problem kernel also refreshes the pair transforms, the multi-CTA ones leave that to
    // k_pair_xform
    PcgOut po;
    po.energy = D.energy + (size_t)k * T.n_prob * PAIREN;
    po.pose = D.pose;
    po.pairM = (D.cluster > 0 || D.coop_grid > 0) ? nullptr : D.pairM;
    const Acc *pen = (const Acc *)D.pairen;
    int pcg_rc = 0;
    run_k(c, BF_K_PCG, [&] {
      if (D.cluster > 0) {
        pcg_rc = launch_pcg_cluster<Acc>(t, D.Df, D.pairoff, D.Minv, (const Acc *)D.rhs, D.x, prm.n_pcg, D.pflags,
                                         D.cluster, T.inc_off.data(), pen, po, c->ex->st);
        return pcg_rc < 0 ? 0 : pcg_rc;
      }
      if (D.coop_grid > 0) {
        pcg_rc = launch_pcg_coop<Acc>(t, D.Df, D.pairoff, D.Minv, (const Acc *)D.rhs, D.x, D.r, D.z, D.p, D.p1, D.q,
                                      prm.n_pcg, D.pflags, D.coop, D.coop_grid, pen, po, mf, c->ex->st);
        return pcg_rc < 0 ? 0 : pcg_rc;
      }
      return launch_pcg<Acc>(t, D.Df, D.pairoff, D.Minv, (const Acc *)D.rhs, D.x, D.r, D.z, D.p, D.q, prm.n_pcg,
                             D.pflags, pen, po, mf, c->ex->st);
    });
    if (pcg_rc < 0) return cuda_fail(c, cudaGetLastError(), "PCG launch");
    if (!po.pairM) run_k(c, BF_K_XFORM, [&] { return launch_pair_xform(t, D.pose, D.pairM, c->ex->st); });
  }
  const double wd = prm.n_gn > 0 ? wdense_at(prm, prm.n_gn - 1) : prm.w_dense;
  record_poses(prm.n_gn);
  linearise<Acc>(c, D, prm, wd, MODE_ENERGY, D.rec ? D.rec + (size_t)prm.n_gn * rec_n : nullptr);
  run_k(c, BF_K_ENERGY, [&] {
    return launch_energy_reduce<Acc>(t, (const Acc *)D.pairen, D.energy + (size_t)prm.n_gn * T.n_prob * PAIREN, c->ex->st);
  });
  CK(cudaGetLastError(), "solve launches");
  return BF_OK;
}

// Capture the GN loop as a CUDA graph, or replay the cached one when everything it depends
// on (table contents, parameters, device buffers) is unchanged.  The tables and initial poses
// have already been uploaded into the workspace by prepare(), which the graph reads.
bf_status run_gn_graph(bf_ctx *c, const HostTables &T, const bf_solve_params &prm, DevSolve &D, bool mixed) {
  // key = parameters, sizes and device buffers, plus the tables (through their generation)
  std::vector<unsigned char> key(sizeof(prm) + 8 * sizeof(int) + 9 * sizeof(void *));
  unsigned char *kp = key.data();
  std::memcpy(kp, &prm, sizeof(prm));
  kp += sizeof(prm);
  const int dims[8] = {T.n_frames, T.n_pairs, T.n_dp, T.n_tiles, T.n_segs, T.n_vars, T.n_prob, mixed ? 1 : 0};
  std::memcpy(kp, dims, sizeof(dims));
  kp += sizeof(dims);
  const void *ptrs[9] = {c->ex->ws, c->A, c->B, c->cP, c->cQ, c->kx, c->ky, (void *)c->ex->st, (void *)c->ex->ws_bytes};
  std::memcpy(kp, ptrs, sizeof(ptrs));
  const bool tables_same = T.gen != 0 && c->ex->graph_gen == T.gen;
  if (c->ex->gexec && tables_same && c->ex->gkey == key) {
    CK(cudaGraphLaunch(c->ex->gexec, c->ex->st), "graph launch");
    c->launches += c->ex->gkernels;
    return BF_OK;
  }
  if (c->ex->gexec) {
    cudaGraphExecDestroy(c->ex->gexec);
    c->ex->gexec = nullptr;
  }
  side_stream(c);  // create the second stream and its events before the capture, not during it
  CK(cudaStreamBeginCapture(c->ex->st, cudaStreamCaptureModeThreadLocal), "begin capture");
  const long long before = c->launches;
  bf_status s = mixed ? run_gn<double>(c, T, prm, D) : run_gn<float>(c, T, prm, D);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->ex->st, &g);
  if (s) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
  c->ex->gexec = ge;
  c->ex->gkey = key;
  c->ex->graph_gen = T.gen;
  c->ex->gkernels = (int)(c->launches - before);
  CK(cudaGraphLaunch(c->ex->gexec, c->ex->st), "graph launch");
  return BF_OK;
}

bf_status check_params(bf_ctx *c, const bf_solve_params *p) {
  if (!p) return fail(c, BF_ERR_INVALID_ARG, "null solve params");
  if (p->n_gn < 0 || p->n_gn > BF_MAX_GN || p->n_pcg < 0 || p->n_pcg > 100000)
    return fail(c, BF_ERR_INVALID_ARG, "n_gn must be in [0, BF_MAX_GN] and n_pcg >= 0");
  if (p->precision != BF_PREC_MIXED && p->precision != BF_PREC_FP32)
    return fail(c, BF_ERR_INVALID_ARG, "unknown precision");
  if (p->precond != BF_PRECOND_BLOCK_JACOBI && p->precond != BF_PRECOND_JACOBI)
    return fail(c, BF_ERR_INVALID_ARG, "unknown preconditioner");
  if (!(p->tau_dist > 0) || !std::isfinite(p->tau_normal) || !std::isfinite(p->max_angle_deg))
    return fail(c, BF_ERR_INVALID_ARG, "bad gates");
  if (p->tile_px < 0 && p->tile_px != BF_TILE_AUTOTUNE)
    return fail(c, BF_ERR_INVALID_ARG, "tile_px must be >= 0 or BF_TILE_AUTOTUNE");
  if (p->pcg_variant < BF_PCG_AUTO || p->pcg_variant > BF_PCG_CLUSTER)
    return fail(c, BF_ERR_INVALID_ARG, "unknown pcg_variant");
  if (!(p->prune_rmax >= 0) || !std::isfinite(p->prune_rmax) || p->prune_rounds < 0 || p->prune_rounds > 100000)
    return fail(c, BF_ERR_INVALID_ARG, "prune_rmax must be finite and >= 0, prune_rounds >= 0");
  if (p->persistent != 0 && p->persistent != 1) return fail(c, BF_ERR_INVALID_ARG, "persistent must be 0 or 1");
  if (p->compensated != 0 && p->compensated != 1) return fail(c, BF_ERR_INVALID_ARG, "compensated must be 0 or 1");
  if (p->compensated && p->persistent)
    return fail(c, BF_ERR_INVALID_ARG, "compensated sums are not available in the persistent launch");
  if (p->dense_tc != 0 && p->dense_tc != 1 && p->dense_tc != 3)
    return fail(c, BF_ERR_INVALID_ARG, "dense_tc must be 0, 1 or 3");
  if (p->dense_tc && (p->persistent || p->compensated))
    return fail(c, BF_ERR_INVALID_ARG, "dense_tc is not available with persistent or compensated");
  if (p->sparse_mode != BF_SPARSE_BLOCKS && p->sparse_mode != BF_SPARSE_MATFREE)
    return fail(c, BF_ERR_INVALID_ARG, "unknown sparse_mode");
  if (p->sparse_mode == BF_SPARSE_MATFREE && p->pcg_variant == BF_PCG_CLUSTER)
    return fail(c, BF_ERR_INVALID_ARG, "the cluster PCG kernel has no matrix-free sparse term");
  return BF_OK;
}

// Solve a set of problems; writes final poses per problem and stats.
// A solve whose device work has been enqueued on an executor's stream.
struct SolveJob {
  HostTables T;
  Exec *ex = nullptr;  // the executor whose table cache T may have come from
  DevSolve D;
  bf_solve_params prm;
  std::vector<int> sizes;  // frames per problem
  size_t n_pose = 0, n_en = 0, o_en = 0, o_vf = 0, o_pf = 0, o_sm = 0, o_sa = 0, o_ce = 0;
  std::chrono::steady_clock::time_point t0;
  bool rec = false;  // the dense evaluations are being recorded (bf_debug_record_association)
};

// Phase 1 (context lock held): build the tables, upload, enqueue the Gauss-Newton loop and the
// asynchronous result copies into the executor's pinned staging.
// ---------------------------------------------------------------- dense work autotuner
// tile_px = BF_TILE_AUTOTUNE: the first solve of a context (per frame size and storage) times the
// dense kernel on its own tables for each candidate decomposition — the target frame staged in
// shared memory when it fits, and tiles of 1, 1/2, 1/4, 1/8 and 1/16 of a frame — takes the
// fastest (median of 3 launches, CUDA events on the solve's stream) and keeps it for the
// context's later solves.  The choice depends on the frame size and storage only, so a problem
// gets the same decomposition alone and inside a batch.
static int tune_tile(bf_ctx *c, const std::vector<Problem> &probs, const bf_solve_params &prm) {
  const int HW = c->cfg.width * c->cfg.height;
  const long long key = ((long long)c->cfg.width << 32) | ((long long)c->cfg.height << 8) | c->cfg.storage;
  auto it = c->tuned_tile.find(key);
  if (it != c->tuned_tile.end()) return it->second;
  std::vector<int> cand;
  if (dense_staged_fits(c->cfg.width, c->cfg.height, c->cfg.storage)) cand.push_back(0);
  for (int d : {1, 2, 4, 8, 16}) {
    const int t = std::max(256, (HW + d - 1) / d);
    if (std::find(cand.begin(), cand.end(), t) == cand.end()) cand.push_back(t);
  }
  int best = cand[0];
  float best_ms = INFINITY;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return best;
  }
  const bool mixed = prm.precision == BF_PREC_MIXED;
  for (int tp : cand) {
    bf_solve_params q = prm;
    q.tile_px = tp;
    HostTables T;
    DevSolve D;
    if (build_tables(c, probs, q, T) || prepare(c, T, 1, mixed ? 8 : 4, false, D, q.pcg_variant)) continue;
    if (T.n_dp == 0) break;  // no dense pairs: nothing to choose
    launch_pair_xform(D.t, D.pose, D.pairM, c->ex->st);
    Gates g;
    g.tau_d2 = (float)(prm.tau_dist * prm.tau_dist);
    g.tau_n = (float)prm.tau_normal;
    std::vector<float> ms;
    for (int r = 0; r < 4; ++r) {
      cudaEventRecord(e0, c->ex->st);
      if (D.t.n_wi > 0) {
        if (mixed) launch_dense_staged<double>(MODE_ACCUM, D.t, frame_store(c), c->intr, D.pairM, g, 1.f, 0.1f,
                                               (double *)D.dpart, D.derr, nullptr, c->ex->st);
        else launch_dense_staged<float>(MODE_ACCUM, D.t, frame_store(c), c->intr, D.pairM, g, 1.f, 0.1f,
                                        (float *)D.dpart, D.derr, nullptr, c->ex->st);
      } else {
        if (mixed) launch_dense<double>(MODE_ACCUM, D.t, frame_store(c), c->intr, D.pairM, g, 1.f, 0.1f,
                                        (double *)D.dpart, nullptr, c->ex->st);
        else launch_dense<float>(MODE_ACCUM, D.t, frame_store(c), c->intr, D.pairM, g, 1.f, 0.1f,
                                 (float *)D.dpart, nullptr, c->ex->st);
      }
      cudaEventRecord(e1, c->ex->st);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) ms.push_back(t);  // the first launch warms up
    }
    std::sort(ms.begin(), ms.end());
    if (!ms.empty() && ms[ms.size() / 2] < best_ms) {
      best_ms = ms[ms.size() / 2];
      best = tp;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  c->tuned_tile[key] = best;
  return best;
}

bf_status enqueue_solve(bf_ctx *c, const std::vector<Problem> &probs, const bf_solve_params &prm_in, SolveJob &J) {
  J.t0 = std::chrono::steady_clock::now();
  J.ex = c->ex;
  bf_solve_params prm = prm_in;
  if (prm.tile_px == BF_TILE_AUTOTUNE) prm.tile_px = tune_tile(c, probs, prm);
  const bool recording = c->assoc_rec && probs.size() == 1 && c->ex == &c->main;
  if (recording) {  // kernel by kernel, so that every dense launch gets its own slab of the record
    prm.use_graph = 0;
    prm.persistent = 0;
  }
  J.prm = prm;
  J.sizes.clear();
  for (const Problem &P : probs) J.sizes.push_back((int)P.ids.size());
  HostTables &T = J.T;
  DevSolve &D = J.D;
  bf_status s = build_tables(c, probs, prm, T);
  if (s) return s;
  const bool mixed = prm.precision == BF_PREC_MIXED;
  const size_t acc_size = mixed ? sizeof(double) : sizeof(float);
  s = prepare(c, T, prm.n_gn, acc_size, false, D, prm.pcg_variant, prm.sparse_mode == BF_SPARSE_MATFREE,
              prm.persistent != 0);
  if (s) return s;
  D.rec = nullptr;
  D.rec_pose = nullptr;
  if (recording) {
    const size_t n_eval = (size_t)prm.n_gn + 1;
    const size_t ni = n_eval * T.n_dp * c->cfg.width * c->cfg.height, nd = n_eval * T.n_frames * 12;
    if (ni > c->rec_dev_n) {
      cudaFree(c->rec_dev);
      c->rec_dev = nullptr;
      c->rec_dev_n = 0;
      CK(cudaMalloc(&c->rec_dev, std::max<size_t>(ni, 1) * sizeof(int)), "association record");
      c->rec_dev_n = ni;
    }
    if (nd > c->rec_pose_n) {
      cudaFree(c->rec_pose_dev);
      c->rec_pose_dev = nullptr;
      c->rec_pose_n = 0;
      CK(cudaMalloc(&c->rec_pose_dev, std::max<size_t>(nd, 1) * sizeof(double)), "pose record");
      c->rec_pose_n = nd;
    }
    D.rec = c->rec_dev;
    D.rec_pose = c->rec_pose_dev;
    J.rec = true;
  }
  if (prm.use_graph && !c->prof) {
    s = run_gn_graph(c, T, prm, D, mixed);
  } else {
    s = mixed ? run_gn<double>(c, T, prm, D) : run_gn<float>(c, T, prm, D);
  }
  if (s) return s;
  J.n_pose = T.pose.size();
  J.n_en = (size_t)(prm.n_gn + 1) * T.n_prob * PAIREN;
  J.o_en = J.n_pose * 8;
  J.o_vf = J.o_en + J.n_en * 8;
  J.o_pf = J.o_vf + 4 * (size_t)T.n_vars;
  J.o_sm = J.o_pf + 4 * (size_t)T.n_prob;
  J.o_sa = J.o_sm + 4 * (size_t)T.n_segs;
  J.o_ce = J.o_sa + 4 * (size_t)T.n_segs;
  s = ensure_pinned(c, J.o_ce + 16);
  if (s) return s;
  unsigned char *pb = c->ex->pin;
  cudaStream_t st = c->ex->st;
  CK(cudaMemcpyAsync(pb, D.pose, J.n_pose * 8, cudaMemcpyDeviceToHost, st), "poses");
  CK(cudaMemcpyAsync(pb + J.o_en, D.energy, J.n_en * 8, cudaMemcpyDeviceToHost, st), "energy");
  if (T.n_vars) CK(cudaMemcpyAsync(pb + J.o_vf, D.vflags, 4 * (size_t)T.n_vars, cudaMemcpyDeviceToHost, st), "flags");
  CK(cudaMemcpyAsync(pb + J.o_pf, D.pflags, 4 * (size_t)T.n_prob, cudaMemcpyDeviceToHost, st), "flags");
  if (T.n_segs) {
    CK(cudaMemcpyAsync(pb + J.o_sm, D.srmax, 4 * (size_t)T.n_segs, cudaMemcpyDeviceToHost, st), "rmax");
    CK(cudaMemcpyAsync(pb + J.o_sa, D.srarg, 4 * (size_t)T.n_segs, cudaMemcpyDeviceToHost, st), "rmax");
  }
  std::memset(pb + J.o_ce, 0, 12);
  if (D.coop_grid > 0)
    CK(cudaMemcpyAsync(pb + J.o_ce, (char *)D.coop + 8, sizeof(int), cudaMemcpyDeviceToHost, st), "pcg status");
  CK(cudaMemcpyAsync(pb + J.o_ce + 4, D.derr, sizeof(int), cudaMemcpyDeviceToHost, st), "dense status");
  if (D.persistent)
    CK(cudaMemcpyAsync(pb + J.o_ce + 8, (char *)D.bq + 8, sizeof(int), cudaMemcpyDeviceToHost, st), "batch status");
  return pin_used(c);
}

// A solve that took its tables from the executor's cache gives them back when it has finished.
static void return_tables(SolveJob &J) {
  if (J.ex == nullptr || !J.ex->tcache) return;
  TableCache &tc = *J.ex->tcache;
  if (tc.lent && J.T.gen != 0 && J.T.gen == tc.gen) {
    tc.T = std::move(J.T);
    tc.lent = false;
  }
}

// Phase 3 (after the executor's stream is synchronised, context lock held): unpack the results.
bf_status finish_solve(bf_ctx *c, SolveJob &J, std::vector<std::vector<Pose12>> &out, bf_solve_stats *stats) {
  const HostTables &T = J.T;
  const bf_solve_params &prm = J.prm;
  const unsigned char *pb = c->ex->pin;
  std::vector<double> pose(J.n_pose), energy(J.n_en);
  std::vector<int> vflags(T.n_vars), pflags(T.n_prob), srarg(T.n_segs);
  std::vector<float> srmax(T.n_segs);
  std::memcpy(pose.data(), pb, J.n_pose * 8);
  std::memcpy(energy.data(), pb + J.o_en, J.n_en * 8);
  if (T.n_vars) std::memcpy(vflags.data(), pb + J.o_vf, 4 * (size_t)T.n_vars);
  std::memcpy(pflags.data(), pb + J.o_pf, 4 * (size_t)T.n_prob);
  if (T.n_segs) {
    std::memcpy(srmax.data(), pb + J.o_sm, 4 * (size_t)T.n_segs);
    std::memcpy(srarg.data(), pb + J.o_sa, 4 * (size_t)T.n_segs);
  }
  int coop_err = 0, dense_err = 0, batch_err = 0;
  std::memcpy(&coop_err, pb + J.o_ce, 4);
  std::memcpy(&dense_err, pb + J.o_ce + 4, 4);
  std::memcpy(&batch_err, pb + J.o_ce + 8, 4);
  if (coop_err) return fail(c, BF_ERR_TIMEOUT, "PCG grid barrier timed out");
  if (batch_err) return fail(c, BF_ERR_TIMEOUT, "persistent batch: a work-queue wait gave up");
  if (dense_err) return fail(c, BF_ERR_TIMEOUT, "dense kernel: frame copy into shared memory timed out");
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - J.t0).count();
  out.assign(T.n_prob, {});
  for (int pi = 0; pi < T.n_prob; ++pi) {
    const int F0 = T.prob_frame0[pi];
    const int n = J.sizes[pi];
    for (int k = 0; k < n; ++k) {
      Pose12 p;
      for (int q = 0; q < 12; ++q) p[q] = pose[(size_t)(F0 + k) * 12 + q];
      out[pi].push_back(p);
    }
    if (!stats) continue;
    bf_solve_stats &S = stats[pi];
    std::memset(&S, 0, sizeof(S));
    S.n_gn_done = prm.n_gn;
    for (int k = 0; k <= prm.n_gn; ++k) {
      const double *e = &energy[((size_t)k * T.n_prob + pi) * PAIREN];
      const double wd = k < prm.n_gn ? wdense_at(prm, k) : (prm.n_gn > 0 ? wdense_at(prm, prm.n_gn - 1) : prm.w_dense);
      S.e_sparse[k] = e[0];
      S.e_photo[k] = e[1];
      S.e_geo[k] = e[2];
      S.n_dense_valid[k] = (long long)llround(e[3]);
      S.energy[k] = prm.w_sparse * e[0] + (prm.dense_on ? wd * (prm.w_photo * e[1] + prm.w_geo * e[2]) : 0.0);
    }
    S.r_max = -1.0;
    S.r_max_pair[0] = S.r_max_pair[1] = -1;
    for (int p = T.prob_pair0[pi]; p < T.prob_pair1[pi]; ++p)
      for (int sg = T.pair_seg0[p]; sg < T.pair_seg1[p]; ++sg)
        if (T.seg_cnt[sg] > 0 && (double)srmax[sg] > S.r_max) {
          S.r_max = srmax[sg];
          S.r_max_pair[0] = T.pair_ida[p];
          S.r_max_pair[1] = T.pair_idb[p];
        }
    S.n_frames = n;
    S.n_pairs = T.prob_npairs[pi];
    S.n_dense_pairs = T.prob_ndense[pi];
    S.n_corr = T.prob_ncorr[pi];
    int fl = pflags[pi];
    for (int v = T.prob_var0[pi]; v < T.prob_var1[pi]; ++v) fl |= vflags[v];
    S.flags = fl;
    S.ms = ms;
  }
  return_tables(J);
  return BF_OK;
}

bf_status solve_once(bf_ctx *c, const std::vector<Problem> &probs, const bf_solve_params &prm,
                     std::vector<std::vector<Pose12>> &out, bf_solve_stats *stats) {
  SolveJob J;
  bf_status s = enqueue_solve(c, probs, prm, J);
  if (s) return s;
  CK(cudaStreamSynchronize(c->ex->st), "solve");
  if (J.rec) {  // the recorded association of every dense evaluation and the poses it used
    const HostTables &T = J.T;
    bf_ctx::AssocRecord &R = c->rec_last;
    R.ids = probs[0].ids;
    R.dp_src.assign(T.dp_src.begin(), T.dp_src.begin() + T.n_dp);
    R.dp_dst.assign(T.dp_dst.begin(), T.dp_dst.begin() + T.n_dp);
    R.n_eval = J.prm.n_gn + 1;
    R.tgt.resize((size_t)R.n_eval * T.n_dp * c->cfg.width * c->cfg.height);
    R.pose.resize((size_t)R.n_eval * T.n_frames * 12);
    CK(cudaMemcpy(R.tgt.data(), c->rec_dev, R.tgt.size() * sizeof(int), cudaMemcpyDeviceToHost), "record");
    CK(cudaMemcpy(R.pose.data(), c->rec_pose_dev, R.pose.size() * sizeof(double), cudaMemcpyDeviceToHost), "record");
  }
  return finish_solve(c, J, out, stats);
}

// Sec. 4.4.1 pruning around the solve: problems whose r_max exceeds prm.prune_rmax lose every
// correspondence of the pair holding it (removed from the context) and are solved again from
// their initial poses, the others keep their result; at most prm.prune_rounds re-solves.
// Afterwards every frame of a problem (but its first) that no remaining pair touches is
// reported invalid.  Without pruning this is one solve.
bf_status solve_problems(bf_ctx *c, const std::vector<Problem> &probs, const bf_solve_params &prm,
                         std::vector<std::vector<Pose12>> &out, bf_solve_stats *stats) {
  if (!(prm.prune_rmax > 0)) {
    bf_status s = solve_once(c, probs, prm, out, stats);
    if (s == BF_OK && stats)
      for (size_t k = 0; k < probs.size(); ++k) stats[k].solves = 1;
    return s;
  }
  const size_t n = probs.size();
  out.assign(n, {});
  std::vector<bf_solve_stats> st(n);
  std::vector<std::vector<std::pair<int, int>>> pruned(n);
  std::vector<int> solves(n, 0);
  std::vector<size_t> active(n);
  for (size_t k = 0; k < n; ++k) active[k] = k;
  const auto t0 = std::chrono::steady_clock::now();
  for (int round = 0; !active.empty(); ++round) {
    std::vector<Problem> sub;
    for (size_t k : active) sub.push_back(probs[k]);
    std::vector<std::vector<Pose12>> sub_out;
    std::vector<bf_solve_stats> sub_st(sub.size());
    bf_status s = solve_once(c, sub, prm, sub_out, sub_st.data());
    if (s) return s;
    std::vector<size_t> next;
    for (size_t q = 0; q < active.size(); ++q) {
      const size_t k = active[q];
      out[k] = sub_out[q];
      st[k] = sub_st[q];
      ++solves[k];
      const bf_solve_stats &S = sub_st[q];
      if (S.r_max > prm.prune_rmax && round < prm.prune_rounds && S.r_max_pair[0] >= 0) {
        corr_erase(c, pair_key(S.r_max_pair[0], S.r_max_pair[1]));
        pruned[k].push_back({S.r_max_pair[0], S.r_max_pair[1]});
        next.push_back(k);
      }
    }
    active.swap(next);
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (size_t k = 0; k < n; ++k) {
    bf_solve_stats &S = st[k];
    S.ms = ms;
    S.solves = solves[k];
    S.n_pruned = (int)pruned[k].size();
    for (int a = 0; a < S.n_pruned && a < BF_MAX_PRUNE; ++a) {
      S.pruned_pairs[2 * a] = pruned[k][a].first;
      S.pruned_pairs[2 * a + 1] = pruned[k][a].second;
    }
    // frames (but the first) without any remaining pair inside the problem
    const std::vector<int> &ids = probs[k].ids;
    S.n_invalid = 0;
    for (size_t a = 1; a < ids.size(); ++a) {
      bool linked = false;
      for (size_t b = 0; b < ids.size() && !linked; ++b) {
        if (b == a) continue;
        auto it = c->corr.find(pair_key(ids[a], ids[b]));
        linked = it != c->corr.end() && !it->second.empty();
      }
      if (!linked) {
        if (S.n_invalid < BF_MAX_PRUNE) S.invalid_frames[S.n_invalid] = ids[a];
        ++S.n_invalid;
      }
    }
    if (stats) stats[k] = S;
  }
  return BF_OK;
}

Pose12 world_of(bf_ctx *c, int id) {
  auto it = c->frames.find(id);
  if (it == c->frames.end()) return ident12();
  const FrameInfo &f = it->second;
  Pose12 w;
  if (f.keyframe_of >= 0 && f.has_world) {
    std::memcpy(w.data(), f.world, sizeof(f.world));
    return w;
  }
  if (f.member_of >= 0) {
    auto ch = c->chunks.find(f.member_of);
    if (ch != c->chunks.end()) {
      const Chunk &C = ch->second;
      for (size_t k = 0; k < C.frames.size(); ++k)
        if (C.frames[k] == id) return compose(world_of(c, C.frames[0]), C.local[k]);
    }
  }
  if (f.has_world) {
    std::memcpy(w.data(), f.world, sizeof(f.world));
    return w;
  }
  return ident12();
}

}  // namespace

// ---------------------------------------------------------------------------- local solves
static bf_status make_local_problems(bf_ctx *c, int n_chunks, const int *chunk_ids, const int *frame_ids,
                                     const int *offsets, const bf_solve_params *params, std::vector<Problem> &probs) {
  probs.assign(n_chunks, Problem());
  for (int k = 0; k < n_chunks; ++k) {
    const int n = offsets[k + 1] - offsets[k];
    if (n < 1) return fail(c, BF_ERR_INVALID_ARG, "local solve: a chunk needs at least one frame");
    Problem &P = probs[k];
    P.ids.assign(frame_ids + offsets[k], frame_ids + offsets[k + 1]);
    P.init.assign(n, ident12());
    if (params->warm_start) {
      auto ch = c->chunks.find(chunk_ids[k]);
      if (ch != c->chunks.end())
        for (int a = 1; a < n; ++a)
          for (size_t b = 0; b < ch->second.frames.size(); ++b)
            if (ch->second.frames[b] == P.ids[a]) P.init[a] = ch->second.local[b];
    }
  }
  return BF_OK;
}

static void commit_local(bf_ctx *c, int n_chunks, const int *chunk_ids, const std::vector<Problem> &probs,
                         const std::vector<std::vector<Pose12>> &out) {
  for (int k = 0; k < n_chunks; ++k) {
    Chunk &C = c->chunks[chunk_ids[k]];
    C.frames = probs[k].ids;
    C.local = out[k];
    c->frames[C.frames[0]].keyframe_of = chunk_ids[k];
    for (size_t a = 1; a < C.frames.size(); ++a) c->frames[C.frames[a]].member_of = chunk_ids[k];
  }
}

static bf_status local_batch(bf_ctx *c, int n_chunks, const int *chunk_ids, const int *frame_ids, const int *offsets,
                             const bf_solve_params *params, bf_solve_stats *stats) {
  std::vector<Problem> probs;
  bf_status s = make_local_problems(c, n_chunks, chunk_ids, frame_ids, offsets, params, probs);
  if (s) return s;
  std::vector<std::vector<Pose12>> out;
  s = solve_problems(c, probs, *params, out, stats);
  if (s) return s;
  commit_local(c, n_chunks, chunk_ids, probs, out);
  return BF_OK;
}

extern "C" bf_status bf_solve_local(bf_ctx *c, int chunk_id, const int *frame_ids, int n,
                                    const bf_solve_params *params, bf_solve_stats *stats) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!frame_ids || n < 1) return fail(c, BF_ERR_INVALID_ARG, "bf_solve_local: bad frame list");
  bf_status s = check_params(c, params);
  if (s) return s;
  const int off[2] = {0, n};
  return local_batch(c, 1, &chunk_id, frame_ids, off, params, stats);
}

extern "C" bf_status bf_solve_local_batch(bf_ctx *c, int n_chunks, const int *chunk_ids, const int *frame_ids,
                                          const int *offsets, const bf_solve_params *params, bf_solve_stats *stats) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (n_chunks < 0 || (n_chunks > 0 && (!chunk_ids || !frame_ids || !offsets)))
    return fail(c, BF_ERR_INVALID_ARG, "bf_solve_local_batch: bad arguments");
  if (n_chunks == 0) return BF_OK;
  bf_status s = check_params(c, params);
  if (s) return s;
  if (offsets[0] != 0) return fail(c, BF_ERR_INVALID_ARG, "bf_solve_local_batch: offsets[0] must be 0");
  return local_batch(c, n_chunks, chunk_ids, frame_ids, offsets, params, stats);
}

// --------------------------------------------------------------------------- global solve
static bf_status make_global_problem(bf_ctx *c, const int *keyframe_ids, int n, Problem &P) {
  P.ids.assign(keyframe_ids, keyframe_ids + n);
  P.init.clear();
  for (int k = 0; k < n; ++k) {
    auto it = c->frames.find(P.ids[k]);
    if (it == c->frames.end()) return fail(c, BF_ERR_NOT_FOUND, "bf_solve_global: unknown keyframe id");
    Pose12 init;
    if (it->second.has_world) {
      std::memcpy(init.data(), it->second.world, sizeof(it->second.world));
    } else if (k == 0) {
      init = ident12();
    } else {
      // previous keyframe's pose composed with the intra-chunk delta linking them (Sec. 4.2)
      init = P.init[k - 1];
      auto pit = c->frames.find(P.ids[k - 1]);
      if (pit != c->frames.end() && pit->second.keyframe_of >= 0) {
        auto ch = c->chunks.find(pit->second.keyframe_of);
        if (ch != c->chunks.end())
          for (size_t b = 0; b < ch->second.frames.size(); ++b)
            if (ch->second.frames[b] == P.ids[k]) init = compose(P.init[k - 1], ch->second.local[b]);
      }
    }
    P.init.push_back(init);
  }
  return BF_OK;
}

static void commit_global(bf_ctx *c, const Problem &P, const std::vector<Pose12> &out) {
  for (size_t k = 0; k < P.ids.size(); ++k) {
    FrameInfo &f = c->frames[P.ids[k]];
    std::memcpy(f.world, out[k].data(), sizeof(f.world));
    f.has_world = true;
  }
}

extern "C" bf_status bf_solve_global(bf_ctx *c, const int *keyframe_ids, int n, const bf_solve_params *params,
                                     bf_solve_stats *stats) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!keyframe_ids || n < 1) return fail(c, BF_ERR_INVALID_ARG, "bf_solve_global: bad keyframe list");
  bf_status s = check_params(c, params);
  if (s) return s;
  Problem P;
  s = make_global_problem(c, keyframe_ids, n, P);
  if (s) return s;
  std::vector<Problem> probs{P};
  std::vector<std::vector<Pose12>> out;
  s = solve_problems(c, probs, *params, out, stats);
  if (s) return s;
  commit_global(c, P, out[0]);
  return BF_OK;
}

extern "C" bf_status bf_get_poses(bf_ctx *c, const int *frame_ids, int n, double *out) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (n < 0 || (n > 0 && (!frame_ids || !out))) return fail(c, BF_ERR_INVALID_ARG, "bf_get_poses: bad arguments");
  for (int k = 0; k < n; ++k) {
    if (!c->frames.count(frame_ids[k])) return fail(c, BF_ERR_NOT_FOUND, "bf_get_poses: unknown frame id");
    to16(world_of(c, frame_ids[k]), out + 16 * k);
  }
  return BF_OK;
}





extern "C" bf_status bf_tuned_tile_px(bf_ctx *c, int *tile_px) {
  if (!c || !tile_px) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  const long long key = ((long long)c->cfg.width << 32) | ((long long)c->cfg.height << 8) | c->cfg.storage;
  auto it = c->tuned_tile.find(key);
  if (it == c->tuned_tile.end()) return fail(c, BF_ERR_NOT_FOUND, "no autotuned decomposition yet");
  *tile_px = it->second;
  return BF_OK;
}

// ------------------------------------------------------------ failure-detection self-test
extern "C" bf_status bf_selftest_wait_timeout(bf_ctx *c, int which, long long limit, int *gave_up) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (which < 0 || which > 2 || limit < 1 || limit > (1LL << 24) || !gave_up)
    return fail(c, BF_ERR_INVALID_ARG, "bf_selftest_wait_timeout: bad arguments");
  cudaStream_t st = c->ex->st;
  int *buf = nullptr;  // [0] the word nothing changes, [1] the kernel's error flag
  bf_status s = dalloc(c, (void **)&buf, 2 * sizeof(int), "self-test");
  if (s) return s;
  cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(int), st);
  int flag = 0;
  if (e == cudaSuccess) {
    launch_selftest_wait(which, (const unsigned *)buf, buf + 1, limit, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(c, buf, 2 * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(c, e, "self-test");
  *gave_up = flag;
  return flag ? fail(c, BF_ERR_TIMEOUT, "self-test: the bounded wait gave up as intended") : BF_OK;
}


// -------------------------------------------------------------------------------- TSDF
extern "C" void bf_default_tsdf_config(bf_tsdf_config *p) {
  if (!p) return;
  p->voxel_size = 0.004;
  p->trunc_voxels = 5;
  p->table_log2 = 20;
  p->max_blocks = 1 << 16;
}

namespace {

void tsdf_release(bf_ctx *c) {
  for (auto &a : c->tsdf_allocs) dfree(c, a.first, a.second);
  c->tsdf_allocs.clear();
  c->tsdf = TsdfDev{};
  c->tsdf_on = false;
  c->tsdf_integrated.clear();
}

TsdfPose tsdf_pose(const Pose12 &T) {
  TsdfPose P;
  for (int k = 0; k < 9; ++k) P.R[k] = (float)T[k];
  for (int k = 0; k < 3; ++k) P.t[k] = (float)T[9 + k];
  return P;
}

// One integrate (+1) or de-integrate (-1) of frame f at pose T; checks the device error bits.
bf_status tsdf_apply(bf_ctx *c, int frame_id, const Pose12 &T, int sign) {
  auto it = c->frames.find(frame_id);
  if (it == c->frames.end()) return fail(c, BF_ERR_NOT_FOUND, "TSDF: unknown frame id");
  cudaStream_t st = c->ex->st;
  CK(cudaMemsetAsync(c->tsdf.err, 0, sizeof(int), st), "TSDF");
  const int call = ++c->tsdf_call;
  run_k(c, BF_K_TSDF, [&] {
    return launch_tsdf(c->tsdf, frame_store(c), c->intr, it->second.slot, tsdf_pose(T), sign, call, st);
  });
  CK(cudaGetLastError(), "TSDF launch");
  int err = 0;
  CK(cudaMemcpyAsync(&err, c->tsdf.err, sizeof(int), cudaMemcpyDeviceToHost, st), "TSDF status");
  CK(cudaStreamSynchronize(st), "TSDF");
  if (err & 8) return fail(c, BF_ERR_INVALID_ARG, "TSDF: a point lies outside the addressable block range");
  if (err) return fail(c, BF_ERR_OUT_OF_MEMORY, "TSDF: hash table or block pool full (raise table_log2 / max_blocks)");
  return BF_OK;
}

// Sec. 5.3 distance: Euler angles R = Rz(g) Ry(b) Rx(a) and translation, weights (2,2,2,1,1,1)
double tsdf_pose_distance(const Pose12 &A, const Pose12 &B) {
  auto eul = [](const Pose12 &T, double *e) {
    e[0] = std::atan2(T[7], T[8]);
    e[1] = std::asin(std::max(-1.0, std::min(1.0, -T[6])));
    e[2] = std::atan2(T[3], T[0]);
  };
  double ea[3], eb[3];
  eul(A, ea);
  eul(B, eb);
  double s = 0.0;
  for (int k = 0; k < 3; ++k) s += (2.0 * ea[k] - 2.0 * eb[k]) * (2.0 * ea[k] - 2.0 * eb[k]);
  for (int k = 0; k < 3; ++k) s += (A[9 + k] - B[9 + k]) * (A[9 + k] - B[9 + k]);
  return std::sqrt(s);
}

}  // namespace

extern "C" bf_status bf_tsdf_init(bf_ctx *c, const bf_tsdf_config *cfg) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!cfg || !(cfg->voxel_size > 0) || !std::isfinite(cfg->voxel_size) || cfg->trunc_voxels < 1 ||
      cfg->trunc_voxels > 64 || cfg->table_log2 < 8 || cfg->table_log2 > 30 || cfg->max_blocks < 1 ||
      cfg->max_blocks > (1 << 29))
    return fail(c, BF_ERR_INVALID_ARG, "bf_tsdf_init: bad configuration");
  CK(cudaStreamSynchronize(c->ex->st), "TSDF init");
  tsdf_release(c);
  const size_t slots = (size_t)1 << cfg->table_log2, nb = (size_t)cfg->max_blocks;
  TsdfDev &v = c->tsdf;
  auto take = [&](void **p, size_t bytes) -> bf_status {
    bf_status s = dalloc(c, p, bytes, "TSDF volume");
    if (!s) c->tsdf_allocs.push_back({*p, bytes});
    return s;
  };
  bf_status s;
  if ((s = take((void **)&v.keys, slots * 8)) || (s = take((void **)&v.vals, slots * 4)) ||
      (s = take((void **)&v.stamp, slots * 4)) || (s = take((void **)&v.touched, nb * 4)) ||
      (s = take((void **)&v.n_touched, 16)) || (s = take((void **)&v.S, nb * 512 * 4)) ||
      (s = take((void **)&v.W, nb * 512 * 4)) || (s = take((void **)&v.SC, nb * 512 * 4))) {
    tsdf_release(c);
    return s;
  }
  v.n_blocks = v.n_touched + 1;
  v.err = v.n_touched + 2;
  cudaStream_t st = c->ex->st;
  CK(cudaMemsetAsync(v.keys, 0xff, slots * 8, st), "TSDF init");
  CK(cudaMemsetAsync(v.vals, 0xff, slots * 4, st), "TSDF init");
  CK(cudaMemsetAsync(v.stamp, 0, slots * 4, st), "TSDF init");
  CK(cudaMemsetAsync(v.n_touched, 0, 16, st), "TSDF init");
  CK(cudaStreamSynchronize(st), "TSDF init");
  v.mask = (unsigned)(slots - 1);
  v.max_blocks = cfg->max_blocks;
  v.K = 2 * cfg->trunc_voxels;  // band samples every half voxel out to mu
  v.h = (float)(0.5 * cfg->voxel_size);
  v.mu = (float)(cfg->trunc_voxels * cfg->voxel_size);
  v.inv_block = (float)(1.0 / (8.0 * cfg->voxel_size));
  v.vs = (float)cfg->voxel_size;
  v.inv_q = (float)1048576.0;
  c->tsdf_cfg = *cfg;
  c->tsdf_on = true;
  c->tsdf_call = 0;
  return BF_OK;
}

extern "C" bf_status bf_tsdf_integrate(bf_ctx *c, int frame_id, const double *pose) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!c->tsdf_on) return fail(c, BF_ERR_INVALID_ARG, "bf_tsdf_integrate: call bf_tsdf_init first");
  if (c->tsdf_integrated.count(frame_id)) return fail(c, BF_ERR_INVALID_ARG, "bf_tsdf_integrate: frame already integrated");
  if (!c->frames.count(frame_id)) return fail(c, BF_ERR_NOT_FOUND, "bf_tsdf_integrate: unknown frame id");
  const Pose12 T = pose ? from16(pose) : world_of(c, frame_id);
  bf_status s = tsdf_apply(c, frame_id, T, +1);
  if (s) return s;
  c->tsdf_integrated[frame_id] = T;
  return BF_OK;
}

extern "C" bf_status bf_tsdf_deintegrate(bf_ctx *c, int frame_id) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->tsdf_integrated.find(frame_id);
  if (!c->tsdf_on || it == c->tsdf_integrated.end())
    return fail(c, BF_ERR_NOT_FOUND, "bf_tsdf_deintegrate: frame not integrated");
  bf_status s = tsdf_apply(c, frame_id, it->second, -1);
  if (s) return s;
  c->tsdf_integrated.erase(it);
  return BF_OK;
}

extern "C" bf_status bf_tsdf_reintegrate(bf_ctx *c, int n_fix, int *frame_ids, int *n_done) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!c->tsdf_on || n_fix < 0) return fail(c, BF_ERR_INVALID_ARG, "bf_tsdf_reintegrate: bad arguments");
  std::vector<std::pair<double, int>> order;  // (-distance, id): descending distance, ties by id
  for (auto &kv : c->tsdf_integrated) {
    const double d = tsdf_pose_distance(kv.second, world_of(c, kv.first));
    if (d > 0) order.push_back({-d, kv.first});
  }
  std::sort(order.begin(), order.end());
  int done = 0;
  for (const auto &o : order) {
    if (done >= n_fix) break;
    const int f = o.second;
    const Pose12 opt = world_of(c, f);
    bf_status s = tsdf_apply(c, f, c->tsdf_integrated[f], -1);
    if (s) return s;
    s = tsdf_apply(c, f, opt, +1);
    if (s) return s;
    c->tsdf_integrated[f] = opt;
    if (frame_ids) frame_ids[done] = f;
    ++done;
  }
  if (n_done) *n_done = done;
  return BF_OK;
}

extern "C" bf_status bf_tsdf_export(bf_ctx *c, long long capacity, int *block_coords, int *sums, long long *n) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!c->tsdf_on || !n || capacity < 0 || (capacity > 0 && (!block_coords || !sums)))
    return fail(c, BF_ERR_INVALID_ARG, "bf_tsdf_export: bad arguments");
  const TsdfDev &v = c->tsdf;
  const size_t slots = (size_t)v.mask + 1;
  cudaStream_t st = c->ex->st;
  std::vector<unsigned long long> keys(slots);
  std::vector<int> vals(slots);
  int nb = 0;
  CK(cudaMemcpyAsync(keys.data(), v.keys, slots * 8, cudaMemcpyDeviceToHost, st), "TSDF export");
  CK(cudaMemcpyAsync(vals.data(), v.vals, slots * 4, cudaMemcpyDeviceToHost, st), "TSDF export");
  CK(cudaMemcpyAsync(&nb, v.n_blocks, sizeof(int), cudaMemcpyDeviceToHost, st), "TSDF export");
  CK(cudaStreamSynchronize(st), "TSDF export");
  std::vector<std::pair<unsigned long long, int>> blocks;
  for (size_t h = 0; h < slots; ++h)
    if (keys[h] != ~0ull && vals[h] >= 0) blocks.push_back({keys[h], vals[h] & ((1 << 30) - 1)});
  std::sort(blocks.begin(), blocks.end());
  *n = (long long)blocks.size();
  const long long m = std::min<long long>(capacity, (long long)blocks.size());
  if (m == 0) return BF_OK;
  nb = std::min(nb, v.max_blocks);
  std::vector<int> S((size_t)nb * 512), W((size_t)nb * 512), SC((size_t)nb * 512);
  CK(cudaMemcpyAsync(S.data(), v.S, S.size() * 4, cudaMemcpyDeviceToHost, st), "TSDF export");
  CK(cudaMemcpyAsync(W.data(), v.W, W.size() * 4, cudaMemcpyDeviceToHost, st), "TSDF export");
  CK(cudaMemcpyAsync(SC.data(), v.SC, SC.size() * 4, cudaMemcpyDeviceToHost, st), "TSDF export");
  CK(cudaStreamSynchronize(st), "TSDF export");
  for (long long k = 0; k < m; ++k) {
    const unsigned long long key = blocks[k].first;
    block_coords[3 * k] = (int)((key >> 42) & 0x1fffff) - (1 << 20);
    block_coords[3 * k + 1] = (int)((key >> 21) & 0x1fffff) - (1 << 20);
    block_coords[3 * k + 2] = (int)(key & 0x1fffff) - (1 << 20);
    const size_t b = (size_t)blocks[k].second * 512;
    std::memcpy(sums + (size_t)k * 1536, S.data() + b, 512 * 4);
    std::memcpy(sums + (size_t)k * 1536 + 512, W.data() + b, 512 * 4);
    std::memcpy(sums + (size_t)k * 1536 + 1024, SC.data() + b, 512 * 4);
  }
  return BF_OK;
}

// ------------------------------------------------------------------- key-point filter
extern "C" void bf_default_keypoint_params(bf_keypoint_params *p) {
  if (!p) return;
  p->max_residual = 0.02;
  p->max_cond = 100.0;
  p->min_area = 0.032;
  p->min_matches = 5;
}

extern "C" bf_status bf_filter_keypoints(bf_ctx *c, int n_pairs, const int *offsets, const float *p_i,
                                         const float *p_j, const bf_keypoint_params *kp, unsigned char *keep,
                                         double *transforms, int *status) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (n_pairs < 0 || (n_pairs > 0 && (!offsets || !keep)) || !kp || !(kp->max_residual >= 0) ||
      !(kp->max_cond >= 1) || !std::isfinite(kp->min_area) || kp->min_matches < 0)
    return fail(c, BF_ERR_INVALID_ARG, "bf_filter_keypoints: bad arguments");
  if (n_pairs == 0) return BF_OK;
  if (offsets[0] != 0) return fail(c, BF_ERR_INVALID_ARG, "bf_filter_keypoints: offsets[0] must be 0");
  for (int k = 0; k < n_pairs; ++k) {
    const int n = offsets[k + 1] - offsets[k];
    if (n < 0 || n > keypoint_nmax())
      return fail(c, BF_ERR_INVALID_ARG, "bf_filter_keypoints: a pair has more than 1024 matches (or a negative count)");
  }
  const long long total = offsets[n_pairs];
  if (total > 0 && (!p_i || !p_j)) return fail(c, BF_ERR_INVALID_ARG, "bf_filter_keypoints: null points");
  // device layout: offsets | p_i | p_j | keep | results
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_off = al(sizeof(int) * (n_pairs + 1)), b_pts = al(12 * (size_t)total),
               b_keep = al((size_t)total), b_res = al(keypoint_result_bytes() * n_pairs);
  const size_t need = b_off + 2 * b_pts + b_keep + b_res;
  cudaStream_t st = c->ex->st;
  if (need > c->kp_cap) {
    CK(cudaStreamSynchronize(st), "key-point buffers");
    dfree(c, c->kp_buf, c->kp_cap);
    c->kp_buf = nullptr;
    c->kp_cap = 0;
    bf_status s = dalloc(c, &c->kp_buf, need, "key-point filter");
    if (s) return s;
    c->kp_cap = need;
  }
  char *base = (char *)c->kp_buf;
  int *d_off = (int *)base;
  float *d_p = (float *)(base + b_off), *d_q = (float *)(base + b_off + b_pts);
  unsigned char *d_keep = (unsigned char *)(base + b_off + 2 * b_pts);
  char *d_res = base + b_off + 2 * b_pts + b_keep;
  CK(cudaMemcpyAsync(d_off, offsets, sizeof(int) * (n_pairs + 1), cudaMemcpyHostToDevice, st), "key-point input");
  if (total > 0) {
    CK(cudaMemcpyAsync(d_p, p_i, 12 * (size_t)total, cudaMemcpyHostToDevice, st), "key-point input");
    CK(cudaMemcpyAsync(d_q, p_j, 12 * (size_t)total, cudaMemcpyHostToDevice, st), "key-point input");
  }
  run_k(c, BF_K_KEYPOINT, [&] {
    return launch_keypoints(n_pairs, d_off, d_p, d_q, kp->max_residual, kp->max_cond, kp->min_matches, kp->min_area,
                            d_keep, d_res, st);
  });
  CK(cudaGetLastError(), "key-point launch");
  std::vector<char> res(keypoint_result_bytes() * n_pairs);
  if (total > 0) CK(cudaMemcpyAsync(keep, d_keep, (size_t)total, cudaMemcpyDeviceToHost, st), "key-point output");
  CK(cudaMemcpyAsync(res.data(), d_res, res.size(), cudaMemcpyDeviceToHost, st), "key-point output");
  CK(cudaStreamSynchronize(st), "key-point filter");
  for (int k = 0; k < n_pairs; ++k) {
    const char *r = res.data() + keypoint_result_bytes() * k;
    double R[9], t[3];
    int stt;
    std::memcpy(R, r, sizeof(R));
    std::memcpy(t, r + sizeof(R), sizeof(t));
    std::memcpy(&stt, r + sizeof(R) + sizeof(t), sizeof(int));
    if (status) status[k] = stt;
    if (transforms) {
      double *m = transforms + 16 * k;
      const double M[16] = {R[0], R[1], R[2], t[0], R[3], R[4], R[5], t[1], R[6], R[7], R[8], t[2], 0, 0, 0, 1};
      if (stt == 0) std::memcpy(m, M, sizeof(M));
      else std::memset(m, 0, sizeof(M));
    }
  }
  return BF_OK;
}

// ----------------------------------------------------------------- dense verification
extern "C" void bf_default_verify_params(bf_verify_params *p) {
  if (!p) return;
  p->tau_dist = 0.15;
  p->tau_normal = 0.9;
  p->tau_color = 0.1;
  p->max_err = 0.075;
  p->min_valid_frac = 0.02;
}

namespace {

// fl32 of a relative transform (R row-major, t) and of its inverse (R^T, -R^T t with the sums
// taken left to right in FP64, then rounded)
void verify_record(const double *R, const double *t, VerifyPair &v) {
  for (int k = 0; k < 9; ++k) v.M[0][k] = (float)R[k];
  for (int a = 0; a < 3; ++a) v.M[0][9 + a] = (float)t[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) v.M[1][3 * a + b] = (float)R[3 * b + a];
  for (int a = 0; a < 3; ++a) {
    const double s = (R[a] * t[0] + R[3 + a] * t[1]) + R[6 + a] * t[2];
    v.M[1][9 + a] = (float)(-s);
  }
}

bool check_verify_params(const bf_verify_params *vp) {
  return vp && vp->tau_dist > 0 && std::isfinite(vp->tau_dist) && std::isfinite(vp->tau_normal) &&
         vp->tau_color > 0 && std::isfinite(vp->tau_color) && std::isfinite(vp->max_err) &&
         std::isfinite(vp->min_valid_frac);
}

// Run the verification kernel over recs; res gets {n_ij, n_ji, e_ij, e_ji} per pair.
bf_status run_verify(bf_ctx *c, const std::vector<VerifyPair> &recs, const bf_verify_params &vp,
                     std::vector<double> &res) {
  const int n = (int)recs.size();
  res.assign(4 * (size_t)n, 0.0);
  if (n == 0) return BF_OK;
  if (n > c->vcap) {
    const int nc = std::max(n, 2 * c->vcap);
    CK(cudaStreamSynchronize(c->ex->st), "verify buffers");
    dfree(c, c->vrec, (size_t)c->vcap * sizeof(VerifyPair));
    dfree(c, c->vout, (size_t)c->vcap * 4 * sizeof(double));
    c->vrec = nullptr;
    c->vout = nullptr;
    c->vcap = 0;
    bf_status s = dalloc(c, (void **)&c->vrec, (size_t)nc * sizeof(VerifyPair), "verification records");
    if (s) return s;
    s = dalloc(c, (void **)&c->vout, (size_t)nc * 4 * sizeof(double), "verification results");
    if (s) return s;
    c->vcap = nc;
  }
  cudaStream_t st = c->ex->st;
  CK(cudaMemcpyAsync(c->vrec, recs.data(), (size_t)n * sizeof(VerifyPair), cudaMemcpyHostToDevice, st),
     "verification records");
  run_k(c, BF_K_VERIFY, [&] {
    return launch_verify(n, c->vrec, frame_store(c), c->intr, (float)(vp.tau_dist * vp.tau_dist),
                         (float)vp.tau_normal, (float)vp.tau_color, c->vout, st);
  });
  CK(cudaGetLastError(), "verification launch");
  CK(cudaMemcpyAsync(res.data(), c->vout, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost, st),
     "verification results");
  CK(cudaStreamSynchronize(st), "verification");
  return BF_OK;
}

double mean_err(const double *r) {
  const double n = r[0] + r[1];
  return n > 0 ? (r[2] + r[3]) / n : INFINITY;
}

}  // namespace

extern "C" bf_status bf_verify_pairs(bf_ctx *c, int n, const int *frame_pairs, const double *rel,
                                     const bf_verify_params *vp, bf_verify_result *out) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (n < 0 || (n > 0 && (!frame_pairs || !rel || !out)) || !check_verify_params(vp))
    return fail(c, BF_ERR_INVALID_ARG, "bf_verify_pairs: bad arguments");
  std::vector<VerifyPair> recs(n);
  for (int k = 0; k < n; ++k) {
    auto fi = c->frames.find(frame_pairs[2 * k]), fj = c->frames.find(frame_pairs[2 * k + 1]);
    if (fi == c->frames.end() || fj == c->frames.end()) return fail(c, BF_ERR_NOT_FOUND, "bf_verify_pairs: unknown frame");
    recs[k].slot_i = fi->second.slot;
    recs[k].slot_j = fj->second.slot;
    const double *m = rel + 16 * k;
    const double R[9] = {m[0], m[1], m[2], m[4], m[5], m[6], m[8], m[9], m[10]};
    const double t[3] = {m[3], m[7], m[11]};
    verify_record(R, t, recs[k]);
  }
  std::vector<double> res;
  bf_status s = run_verify(c, recs, *vp, res);
  if (s) return s;
  const double need = vp->min_valid_frac * c->cfg.width * c->cfg.height;
  for (int k = 0; k < n; ++k) {
    const double *r = &res[4 * (size_t)k];
    bf_verify_result &o = out[k];
    o.n_ij = (int)r[0];
    o.n_ji = (int)r[1];
    o.err_ij = r[2];
    o.err_ji = r[3];
    o.mean_err = mean_err(r);
    o.valid = (r[0] + r[1] >= need && o.mean_err <= vp->max_err) ? 1 : 0;
  }
  return BF_OK;
}

extern "C" bf_status bf_validate_chunk(bf_ctx *c, int chunk_id, double max_err, const bf_verify_params *vp,
                                       int *valid, double *worst_err, int *worst_pair) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!valid || !check_verify_params(vp) || !std::isfinite(max_err))
    return fail(c, BF_ERR_INVALID_ARG, "bf_validate_chunk: bad arguments");
  auto ch = c->chunks.find(chunk_id);
  if (ch == c->chunks.end()) return fail(c, BF_ERR_NOT_FOUND, "bf_validate_chunk: unknown chunk (not solved yet)");
  const Chunk &C = ch->second;
  const int n = (int)C.frames.size();
  std::vector<VerifyPair> recs;
  std::vector<std::pair<int, int>> ids;
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      // T_b^-1 T_a of the local poses, entries summed left to right in FP64
      const Pose12 &Ti = C.local[a], &Tj = C.local[b];
      double R[9], t[3];
      const double d[3] = {Ti[9] - Tj[9], Ti[10] - Tj[10], Ti[11] - Tj[11]};
      for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) R[3 * r + q] = (Tj[r] * Ti[q] + Tj[3 + r] * Ti[3 + q]) + Tj[6 + r] * Ti[6 + q];
        t[r] = (Tj[r] * d[0] + Tj[3 + r] * d[1]) + Tj[6 + r] * d[2];
      }
      VerifyPair v;
      v.slot_i = c->frames[C.frames[a]].slot;
      v.slot_j = c->frames[C.frames[b]].slot;
      verify_record(R, t, v);
      recs.push_back(v);
      ids.push_back({C.frames[a], C.frames[b]});
    }
  std::vector<double> res;
  bf_status s = run_verify(c, recs, *vp, res);
  if (s) return s;
  double worst = 0.0;
  int wa = -1, wb = -1;
  for (size_t k = 0; k < recs.size(); ++k) {
    const double *r = &res[4 * k];
    if (r[0] + r[1] > 0 && mean_err(r) > worst) {
      worst = mean_err(r);
      wa = ids[k].first;
      wb = ids[k].second;
    }
  }
  *valid = worst <= max_err ? 1 : 0;
  if (worst_err) *worst_err = worst;
  if (worst_pair) {
    worst_pair[0] = wa;
    worst_pair[1] = wb;
  }
  return BF_OK;
}

// ---------------------------------------------------------------------- system inspection
template <typename Acc>
static bf_status build_system_t(bf_ctx *c, const HostTables &T, DevSolve &D, const bf_solve_params &prm, double *A,
                                double *b, double *energy4, long long *n_dense) {
  run_k(c, BF_K_XFORM, [&] { return launch_pair_xform(D.t, D.pose, D.pairM, c->ex->st); });
  linearise<Acc>(c, D, prm, prm.w_dense, MODE_ACCUM);
  run_k(c, BF_K_ENERGY, [&] { return launch_energy_reduce<Acc>(D.t, (const Acc *)D.pairen, D.energy, c->ex->st); });
  run_k(c, BF_K_ASSEMBLE, [&] {
    return launch_assemble<Acc>(D.t, (const Acc *)D.pairblk, prm.precond, (Acc *)D.Dd, (Acc *)D.rhs, D.Df, D.Minv,
                                D.vflags, c->ex->st);
  });
  CK(cudaGetLastError(), "build system launches");
  std::vector<Acc> Dd((size_t)T.n_vars * 36), rhs((size_t)T.n_vars * 6), pb((size_t)T.n_pairs * PAIRBLK);
  double en[PAIREN];
  if (T.n_vars) {
    CK(cudaMemcpyAsync(Dd.data(), D.Dd, Dd.size() * sizeof(Acc), cudaMemcpyDeviceToHost, c->ex->st), "Dd");
    CK(cudaMemcpyAsync(rhs.data(), D.rhs, rhs.size() * sizeof(Acc), cudaMemcpyDeviceToHost, c->ex->st), "rhs");
  }
  if (T.n_pairs) CK(cudaMemcpyAsync(pb.data(), D.pairblk, pb.size() * sizeof(Acc), cudaMemcpyDeviceToHost, c->ex->st), "pb");
  CK(cudaMemcpyAsync(en, D.energy, sizeof(en), cudaMemcpyDeviceToHost, c->ex->st), "energy");
  CK(cudaStreamSynchronize(c->ex->st), "build system");
  const int m = 6 * T.n_vars;
  std::fill(A, A + (size_t)m * m, 0.0);
  for (int v = 0; v < T.n_vars; ++v) {
    for (int i = 0; i < 6; ++i) {
      b[6 * v + i] = (double)rhs[6 * v + i];
      for (int j = 0; j < 6; ++j) A[(size_t)(6 * v + i) * m + 6 * v + j] = (double)Dd[36 * v + 6 * i + j];
    }
  }
  for (int p = 0; p < T.n_pairs; ++p) {
    const int va = T.frame_var[T.pair_a[p]], vb = T.frame_var[T.pair_b[p]];
    if (va < 0 || vb < 0) continue;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        const double x = (double)pb[(size_t)p * PAIRBLK + PB_AB + 6 * i + j];
        A[(size_t)(6 * va + i) * m + 6 * vb + j] += x;
        A[(size_t)(6 * vb + j) * m + 6 * va + i] += x;
      }
  }
  energy4[1] = en[0];
  energy4[2] = en[1];
  energy4[3] = en[2];
  energy4[0] = prm.w_sparse * en[0] + (prm.dense_on ? prm.w_dense * (prm.w_photo * en[1] + prm.w_geo * en[2]) : 0.0);
  if (n_dense) *n_dense = (long long)llround(en[3]);
  return BF_OK;
}

extern "C" bf_status bf_build_system(bf_ctx *c, const int *frame_ids, int n, const double *poses,
                                     const bf_solve_params *params, double *A, double *b, double *energy4,
                                     long long *n_dense) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!frame_ids || n < 1 || !poses || !A || !b || !energy4)
    return fail(c, BF_ERR_INVALID_ARG, "bf_build_system: bad arguments");
  bf_status s = check_params(c, params);
  if (s) return s;
  Problem P;
  P.ids.assign(frame_ids, frame_ids + n);
  for (int k = 0; k < n; ++k) P.init.push_back(from16(poses + 16 * k));
  HostTables T;
  s = build_tables(c, {P}, *params, T);
  if (s) return s;
  const bool mixed = params->precision == BF_PREC_MIXED;
  DevSolve D;
  s = prepare(c, T, 0, mixed ? 8 : 4, false, D);
  if (s) return s;
  return mixed ? build_system_t<double>(c, T, D, *params, A, b, energy4, n_dense)
               : build_system_t<float>(c, T, D, *params, A, b, energy4, n_dense);
}

extern "C" bf_status bf_debug_association(bf_ctx *c, int frame_i, int frame_j, const double *pose_i,
                                          const double *pose_j, const bf_solve_params *params, int32_t *out_target) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (!pose_i || !pose_j || !out_target || frame_i == frame_j)
    return fail(c, BF_ERR_INVALID_ARG, "bf_debug_association: bad arguments");
  bf_status s = check_params(c, params);
  if (s) return s;
  auto fi = c->frames.find(frame_i), fj = c->frames.find(frame_j);
  if (fi == c->frames.end() || fj == c->frames.end()) return fail(c, BF_ERR_NOT_FOUND, "unknown frame id");
  const int HW = c->cfg.width * c->cfg.height;
  HostTables T;
  T.n_frames = 2;
  T.n_pairs = 1;
  T.n_dp = 1;
  T.n_prob = 1;
  T.frame_slot = {fi->second.slot, fj->second.slot};
  T.frame_var = {-1, -1};
  T.pair_a = {0};
  T.pair_b = {1};
  T.pair_dp = {0, -1};
  T.pair_seg0 = {0};
  T.pair_seg1 = {0};
  T.dp_src = {0};
  T.dp_dst = {1};
  T.dp_pair = {0};
  T.dp_dir = {0};
  T.dp_tile0 = {0};
  const int tile_px = params->tile_px > 0 ? params->tile_px : std::min(HW, 4800);
  for (int px = 0; px < HW; px += tile_px) {
    T.tile_dp.push_back(0);
    T.tile_px0.push_back(px);
    T.tile_px1.push_back(std::min(HW, px + tile_px));
    ++T.n_tiles;
  }
  T.dp_tile1 = {T.n_tiles};
  T.n_vars = 0;
  T.inc_off = {0};
  T.prob_var0 = {0};
  T.prob_var1 = {0};
  T.prob_pair0 = {0};
  T.prob_pair1 = {1};
  T.prob_tile0 = {0};
  T.prob_tile1 = {T.n_tiles};
  T.prob_seg0 = {0};
  T.prob_seg1 = {0};
  const Pose12 a = from16(pose_i), b = from16(pose_j);
  T.pose.assign(a.begin(), a.end());
  T.pose.insert(T.pose.end(), b.begin(), b.end());
  DevSolve D;
  s = prepare(c, T, 0, 4, true, D);
  if (s) return s;
  Gates g;
  g.tau_d2 = (float)(params->tau_dist * params->tau_dist);
  g.tau_n = (float)params->tau_normal;
  run_k(c, BF_K_XFORM, [&] { return launch_pair_xform(D.t, D.pose, D.pairM, c->ex->st); });
  run_k(c, BF_K_DENSE, [&] {
    return launch_dense<float>(MODE_ASSOC, D.t, frame_store(c), c->intr, D.pairM, g, 0.f, 0.f, nullptr, D.assoc,
                               c->ex->st);
  });
  CK(cudaGetLastError(), "association launch");
  CK(cudaMemcpyAsync(out_target, D.assoc, HW * sizeof(int), cudaMemcpyDeviceToHost, c->ex->st), "association");
  CK(cudaStreamSynchronize(c->ex->st), "association");
  return BF_OK;
}

extern "C" bf_status bf_debug_record_association(bf_ctx *c, int enable) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  c->assoc_rec = enable != 0;
  if (!c->assoc_rec) {
    cudaFree(c->rec_dev);
    cudaFree(c->rec_pose_dev);
    cudaGetLastError();
    c->rec_dev = nullptr;
    c->rec_pose_dev = nullptr;
    c->rec_dev_n = c->rec_pose_n = 0;
    c->rec_last = bf_ctx::AssocRecord();
  }
  return BF_OK;
}

extern "C" bf_status bf_debug_recorded_association(bf_ctx *c, int eval, int frame_i, int frame_j,
                                                   int32_t *out_target, double *pose_i, double *pose_j) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  const bf_ctx::AssocRecord &R = c->rec_last;
  if (!out_target) return fail(c, BF_ERR_INVALID_ARG, "bf_debug_recorded_association: null output");
  if (R.n_eval == 0) return fail(c, BF_ERR_NOT_FOUND, "bf_debug_recorded_association: nothing recorded");
  if (eval < 0 || eval >= R.n_eval)
    return fail(c, BF_ERR_INVALID_ARG, "bf_debug_recorded_association: evaluation index out of range");
  const int n = (int)R.ids.size(), n_dp = (int)R.dp_src.size();
  int li = -1, lj = -1;
  for (int k = 0; k < n; ++k) {
    if (R.ids[k] == frame_i) li = k;
    if (R.ids[k] == frame_j) lj = k;
  }
  int d = -1;
  for (int k = 0; k < n_dp && li >= 0 && lj >= 0; ++k)
    if (R.dp_src[k] == li && R.dp_dst[k] == lj) d = k;
  if (d < 0) return fail(c, BF_ERR_NOT_FOUND, "bf_debug_recorded_association: pair not in the recorded solve");
  const size_t HW = (size_t)c->cfg.width * c->cfg.height;
  std::memcpy(out_target, R.tgt.data() + ((size_t)eval * n_dp + d) * HW, HW * sizeof(int32_t));
  auto pose16 = [&](int l, double *o) {
    const double *p = R.pose.data() + ((size_t)eval * n + l) * 12;
    const double m[16] = {p[0], p[1], p[2], p[9], p[3], p[4], p[5], p[10], p[6], p[7], p[8], p[11], 0, 0, 0, 1};
    std::memcpy(o, m, sizeof(m));
  };
  if (pose_i) pose16(li, pose_i);
  if (pose_j) pose16(lj, pose_j);
  return BF_OK;
}

// ------------------------------------------------------------------------------- serving
// Continuous batching on a persistent context.  A worker slot takes the request at the head of
// the queue and, for local solves, every following local request with identical parameters (up
// to max_batch): the batch is one bf_solve_local_batch problem set.  It enqueues the batch on
// its own stream under the context lock, waits for the GPU without the lock (other slots form
// and launch their batches meanwhile, so batches overlap on the device), then unpacks results
// under the lock.  Admission: a batch whose solve workspace would exceed the context's HBM budget
// is halved and the rest returned to the queue head; a single request that cannot fit fails with
// BF_ERR_OUT_OF_MEMORY.
static void complete_requests(Server &S, const std::vector<uint64_t> &batch, bf_status st,
                              const std::vector<bf_solve_stats> *stats) {
  std::lock_guard<std::mutex> q(S.qm);
  const auto now = std::chrono::steady_clock::now();
  for (size_t k = 0; k < batch.size(); ++k) {
    auto it = S.reqs.find(batch[k]);
    if (it == S.reqs.end()) continue;
    ServeReq &r = it->second;
    r.done = true;
    r.status = st;
    if (stats && k < stats->size()) r.stats = (*stats)[k];
    r.stats.ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
  }
  S.dcv.notify_all();
}

static void run_batch(bf_ctx *c, Exec &ex, std::vector<uint64_t> batch) {
  Server &S = *c->srv;
  while (!batch.empty()) {
    std::vector<Problem> probs;
    std::vector<int> chunk_ids;
    bf_solve_params prm{};
    int kind = 0;
    {
      std::lock_guard<std::mutex> q(S.qm);
      const ServeReq &h = S.reqs[batch[0]];
      kind = h.kind;
      prm = h.prm;
    }
    std::unique_lock<std::mutex> lk(c->mu);
    // chunk solves run on the slot's high-priority stream, global solves on its low-priority one:
    // when both kinds are resident the scheduler dispatches the short chunk kernels first
    ex.st = kind == BF_REQ_GLOBAL ? ex.st_lo : ex.st_hi;
    c->ex = &ex;
    bf_status st = check_params(c, &prm);
    if (!st) {
      if (cudaStreamWaitEvent(ex.st, c->data_ev, 0) != cudaSuccess) {
        cudaGetLastError();
        st = BF_ERR_CUDA;
      }
    }
    if (!st) {
      std::lock_guard<std::mutex> q(S.qm);
      if (kind == BF_REQ_GLOBAL) {
        const ServeReq &r = S.reqs[batch[0]];
        Problem P;
        st = make_global_problem(c, r.ids.data(), (int)r.ids.size(), P);
        probs.push_back(P);
      } else {
        std::vector<int> flat, offs{0};
        for (uint64_t t : batch) {
          const ServeReq &r = S.reqs[t];
          flat.insert(flat.end(), r.ids.begin(), r.ids.end());
          offs.push_back((int)flat.size());
          chunk_ids.push_back(r.chunk_id);
        }
        st = make_local_problems(c, (int)batch.size(), chunk_ids.data(), flat.data(), offs.data(), &prm, probs);
      }
    }
    SolveJob J;
    if (!st) st = enqueue_solve(c, probs, prm, J);
    if (st == BF_ERR_OUT_OF_MEMORY && batch.size() > 1) {
      // admission: return the second half to the head of the queue and retry with the first
      c->ex = &c->main;
      lk.unlock();
      const size_t half = batch.size() / 2;
      {
        std::lock_guard<std::mutex> q(S.qm);
        for (size_t k = batch.size(); k-- > half;) S.pending.push_front(batch[k]);
        S.qcv.notify_one();
      }
      batch.resize(half);
      continue;
    }
    if (st) {
      c->ex = &c->main;
      lk.unlock();
      complete_requests(S, batch, st, nullptr);
      return;
    }
    ++c->in_flight;
    c->ex = &c->main;
    lk.unlock();
    const cudaError_t e = cudaStreamSynchronize(ex.st);
    lk.lock();
    c->ex = &ex;
    std::vector<bf_solve_stats> stats(probs.size());
    std::vector<std::vector<Pose12>> out;
    st = e != cudaSuccess ? cuda_fail(c, e, "serving batch") : finish_solve(c, J, out, stats.data());
    if (!st) {
      if (kind == BF_REQ_GLOBAL)
        commit_global(c, probs[0], out[0]);
      else
        commit_local(c, (int)probs.size(), chunk_ids.data(), probs, out);
    }
    --c->in_flight;
    c->ex = &c->main;
    c->busy_cv.notify_all();
    lk.unlock();
    complete_requests(S, batch, st, &stats);
    return;
  }
}

static void serve_worker(bf_ctx *c, int slot) {
  cudaSetDevice(c->cfg.device);
  Server &S = *c->srv;
  Exec &ex = *S.slots[slot];
  for (;;) {
    std::vector<uint64_t> batch;
    {
      std::unique_lock<std::mutex> q(S.qm);
      S.qcv.wait(q, [&] { return S.stop || !S.pending.empty(); });
      if (S.stop) return;
      const uint64_t h = S.pending.front();
      S.pending.pop_front();
      batch.push_back(h);
      const ServeReq &hr = S.reqs[h];
      if (hr.kind == BF_REQ_LOCAL) {
        while (!S.pending.empty() && (int)batch.size() < S.max_batch) {
          const ServeReq &nr = S.reqs[S.pending.front()];
          if (nr.kind != BF_REQ_LOCAL || std::memcmp(&nr.prm, &hr.prm, sizeof(bf_solve_params)) != 0) break;
          batch.push_back(S.pending.front());
          S.pending.pop_front();
        }
      }
    }
    run_batch(c, ex, batch);
  }
}

extern "C" bf_status bf_serve_start(bf_ctx *c, int n_slots, int max_batch, int max_queue) {
  if (!c) return BF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  if (c->srv) return fail(c, BF_ERR_INVALID_ARG, "bf_serve_start: already serving");
  if (n_slots < 1 || n_slots > 8 || max_batch < 1 || max_queue < 1)
    return fail(c, BF_ERR_INVALID_ARG, "bf_serve_start: need 1 <= n_slots <= 8, max_batch >= 1, max_queue >= 1");
  std::unique_ptr<Server> S(new Server());
  S->max_batch = max_batch;
  S->max_queue = max_queue;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    cudaGetLastError();
    least = greatest = 0;
  }
  for (int k = 0; k < n_slots; ++k) {
    std::unique_ptr<Exec> e(new Exec());
    if (cudaStreamCreateWithPriority(&e->st_hi, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&e->st_lo, cudaStreamNonBlocking, least) != cudaSuccess) {
      cudaGetLastError();
      if (e->st_hi) cudaStreamDestroy(e->st_hi);
      for (auto &x : S->slots) {
        cudaStreamDestroy(x->st_hi);
        cudaStreamDestroy(x->st_lo);
      }
      return fail(c, BF_ERR_CUDA, "bf_serve_start: stream creation failed");
    }
    e->st = e->st_hi;
    S->slots.push_back(std::move(e));
  }
  c->srv = std::move(S);
  for (int k = 0; k < n_slots; ++k) c->srv->workers.emplace_back(serve_worker, c, k);
  return BF_OK;
}

extern "C" bf_status bf_serve_stop(bf_ctx *c) {
  if (!c || !c->srv) return BF_OK;
  Server &S = *c->srv;
  {
    std::lock_guard<std::mutex> q(S.qm);
    S.stop = true;
    S.qcv.notify_all();
  }
  for (auto &t : S.workers) t.join();
  std::vector<uint64_t> cancelled;
  {
    std::lock_guard<std::mutex> q(S.qm);
    cancelled.assign(S.pending.begin(), S.pending.end());
    S.pending.clear();
  }
  complete_requests(S, cancelled, BF_ERR_BUSY, nullptr);
  std::unique_lock<std::mutex> lk(c->mu);
  for (auto &e : S.slots) {
    cudaStreamSynchronize(e->st_hi);
    cudaStreamSynchronize(e->st_lo);
    free_exec(c, *e);
    cudaStreamDestroy(e->st_hi);
    cudaStreamDestroy(e->st_lo);
  }
  cudaGetLastError();
  c->srv.reset();
  return BF_OK;
}

extern "C" bf_status bf_submit(bf_ctx *c, const bf_request *req, uint64_t *ticket) {
  if (!c || !req || !ticket) return BF_ERR_INVALID_ARG;
  if (!c->srv) return BF_ERR_INVALID_ARG;
  if ((req->kind != BF_REQ_LOCAL && req->kind != BF_REQ_GLOBAL) || !req->frame_ids || req->n < 1)
    return BF_ERR_INVALID_ARG;
  if (req->params.prune_rmax != 0.0) return BF_ERR_INVALID_ARG;  // pruning re-solves: synchronous API only
  Server &S = *c->srv;
  std::lock_guard<std::mutex> q(S.qm);
  if ((int)S.pending.size() >= S.max_queue) return BF_ERR_BUSY;
  const uint64_t t = S.next_ticket++;
  ServeReq &r = S.reqs[t];
  r.kind = req->kind;
  r.chunk_id = req->chunk_id;
  r.ids.assign(req->frame_ids, req->frame_ids + req->n);
  r.prm = req->params;
  r.prm.use_graph = 0;  // batches differ from one another: no graph reuse
  r.t_submit = std::chrono::steady_clock::now();
  S.pending.push_back(t);
  S.qcv.notify_one();
  *ticket = t;
  return BF_OK;
}

extern "C" bf_status bf_wait(bf_ctx *c, uint64_t ticket, int timeout_ms, bf_solve_stats *stats) {
  if (!c || !c->srv) return BF_ERR_INVALID_ARG;
  Server &S = *c->srv;
  std::unique_lock<std::mutex> q(S.qm);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return BF_ERR_NOT_FOUND;
  auto ready = [&] {
    auto jt = S.reqs.find(ticket);
    return jt == S.reqs.end() || jt->second.done;
  };
  if (timeout_ms < 0)
    S.dcv.wait(q, ready);
  else if (!S.dcv.wait_for(q, std::chrono::milliseconds(timeout_ms), ready))
    return BF_ERR_TIMEOUT;
  it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return BF_ERR_NOT_FOUND;
  const bf_status st = it->second.status;
  if (stats) *stats = it->second.stats;
  S.reqs.erase(it);
  return st;
}
