// Query server: continuous batching of single-source traversals over a pool
// of device-resident graphs (C ABI in include/s3bfs.h, bfs_server_*).
//
// Host side of the scheduler.  Each bfs_server_poll() call
//   1. admits queued queries, in arrival order, while a slot is free and the
//      query's working memory fits in the server's device arena (admission by
//      free memory), and initialises them (level 0);
//   2. makes one cooperative launch of k_serve, which advances every running
//      query level by level (several queries share the grid) until one of
//      them finishes or a level budget is spent;
//   3. retires the finished queries: their outputs are translated or copied
//      where needed and their memory returns to the arena.
// Queries that arrive while others run join at the next launch, so their
// levels overlap on the device with those already running.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "host_internal.h"
#include "serve_device.cuh"

using namespace s3bfs;

// a0 for one query, and the slot's copy of its level-0 sizes
__global__ void __launch_bounds__(256) k_serve_init(Params p, SlotDev* sd) {
  init_traversal(p, 0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sd->n = 1;
    sd->e = p.row_ptr[p.src + 1] - p.row_ptr[p.src];
  }
}

static const void* serve_fn(int wpc) {
  return wpc == 32 ? (const void*)k_serve<32> : wpc == 16 ? (const void*)k_serve<16> : (const void*)k_serve<8>;
}

__global__ void __launch_bounds__(256) k_serve_finalize(int32_t n, const int32_t* inv, const int32_t* perm,
                                                        const int32_t* level, const int32_t* parent,
                                                        int32_t* level_out, int32_t* parent_out) {
  finalize_outputs(n, inv, perm, level, parent, level_out, parent_out, n, -1);  // the server clears every entry
}

namespace {

double now_us() {
  using namespace std::chrono;
  return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over one device region; free blocks coalesce.
struct Arena {
  char* base = nullptr;
  size_t bytes = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  void init(char* b, size_t n) {
    base = b;
    bytes = n;
    free_blocks.clear();
    free_blocks[0] = n;
  }
  bool alloc(size_t n, size_t* off) {
    n = align256(n);
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, o = it->first + n;
        free_blocks.erase(it);
        if (rest) free_blocks[o] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = align256(n);
    auto it = free_blocks.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (const auto& kv : free_blocks) m = std::max(m, kv.second);
    return m;
  }
};

struct Query {
  int64_t tag = 0;
  int32_t graph = 0, src = 0;
  int32_t* level_out = nullptr;
  int32_t* parent_out = nullptr;
  bool lvl_dev = false, par_dev = false;
  double t_submit = 0, t_admit = 0;
  size_t arena_off = 0, arena_bytes = 0;
  int32_t* level = nullptr;   // working arrays (the caller's device buffers when possible)
  int32_t* parent = nullptr;
  int32_t* stage = nullptr;   // 2 n for translated outputs bound for host buffers
};

}  // namespace

struct bfs_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  // 16-warp CTAs, one per SM: p99 64.7 against 76.3 ms with 8-warp ones on the
  // 32-graph pool at 0.7 load (the deep grids' levels pay fewer barrier arrivals)
  int sms = 0, wpc = 16, ctas = 0;
  int nslots = 64, levels_per_launch = 64, grain = 64;
  int local_levels = 0;
  long long spin_ns = 1000000000ll;
  std::vector<bfs_graph*> graphs;
  Arena arena;
  void* d_arena = nullptr;
  SlotDev* d_slots = nullptr;
  SlotDev* h_slots = nullptr;      // pinned mirror
  DevState* d_slot_st = nullptr;   // one per slot
  ChunkStatus* d_slot_status = nullptr;  // ctas per slot
  DevState* d_st = nullptr;        // the server's barrier / error state
  int32_t* d_arrive = nullptr;
  int32_t* d_finished = nullptr;
  volatile int32_t* h_wake = nullptr;  // pinned, mapped: set by submissions
  int32_t* d_wake = nullptr;           // its device address
  bool polling = false;                // a poll is in progress (one poller at a time)
  DevState* h_st = nullptr;        // pinned
  std::vector<Query> running;      // by slot
  std::vector<bool> busy;
  std::deque<Query> queue;
  std::deque<bfs_completion> done;
  std::vector<void*> allocs;
  std::mutex mu;
};

static int sdalloc(bfs_server* s, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(BFS_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  s->allocs.push_back(*p);
  return BFS_OK;
}

extern "C" void bfs_server_destroy(bfs_server* s) {
  if (!s) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_slots) cudaFreeHost(s->h_slots);
  if (s->h_st) cudaFreeHost(s->h_st);
  if (s->h_wake) cudaFreeHost(const_cast<int32_t*>(s->h_wake));
  cudaSetDevice(cur);
  delete s;
}

// working memory of one query in the arena
static size_t query_bytes(const bfs_graph* g, bool internal_out, bool stage) {
  const size_t n = (size_t)g->n, m = (size_t)g->nnz;
  size_t b = 6 * align256(sizeof(int32_t) * (n + 4));               // F, RS, EX x 2
  b += align256(sizeof(int2) * (m + 32)) + align256(sizeof(int32_t) * (m + 32));  // candidates
  if (internal_out) b += 2 * align256(sizeof(int32_t) * (n + 4));   // level, parent
  if (stage) b += 2 * align256(sizeof(int32_t) * (n + 4));
  return b;
}

static int server_create_impl(bfs_server* s, bfs_graph* const* graphs, int32_t ngraphs,
                              const bfs_server_opts* opts) {
  CUDA_TRY(cudaGetDevice(&s->device));
  CUDA_TRY(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device));
  for (int i = 0; i < ngraphs; ++i) {
    if (!graphs[i]) return fail(BFS_E_INVAL, "graph %d is NULL", i);
    if (graphs[i]->device != s->device) return fail(BFS_E_INVAL, "graph %d is on another device", i);
    s->graphs.push_back(graphs[i]);
  }
  size_t arena_bytes = 0;
  if (opts) {
    if (opts->slots > 0) s->nslots = opts->slots;
    if (opts->levels_per_launch > 0) s->levels_per_launch = opts->levels_per_launch;
    if (opts->chunk_edges > 0) s->grain = opts->chunk_edges;
    if (opts->cta_warps != 0) s->wpc = opts->cta_warps;
    if (opts->spin_limit_ms > 0) s->spin_ns = (long long)opts->spin_limit_ms * 1000000ll;
    if (opts->arena_bytes > 0) arena_bytes = (size_t)opts->arena_bytes;
    if (opts->local_levels > 0) s->local_levels = opts->local_levels;
  }
  if (s->nslots > kMaxSlots) return fail(BFS_E_INVAL, "slots = %d: at most %d", s->nslots, kMaxSlots);
  if (s->wpc != 8 && s->wpc != 16 && s->wpc != 32) return fail(BFS_E_INVAL, "cta_warps = %d: use 8, 16 or 32", s->wpc);
  const void* fn = serve_fn(s->wpc);
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, s->wpc * kWarp, 0));
  if (per_sm < 1) return fail(BFS_E_CUDA, "serving kernel cannot be resident (occupancy 0)");
  s->ctas = per_sm * s->sms;
  if (s->nslots > s->ctas) s->nslots = s->ctas;  // every running query needs a CTA
  if (arena_bytes == 0) {
    size_t fr = 0, tot = 0;
    CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    arena_bytes = std::min<size_t>(fr / 2, (size_t)32 << 30);
  }
  int rc;
  if ((rc = sdalloc(s, &s->d_arena, arena_bytes)) != BFS_OK) return rc;
  s->arena.init(static_cast<char*>(s->d_arena), arena_bytes);
  void* p;
  if ((rc = sdalloc(s, &p, sizeof(SlotDev) * (size_t)s->nslots)) != BFS_OK) return rc;
  s->d_slots = static_cast<SlotDev*>(p);
  if ((rc = sdalloc(s, &p, sizeof(DevState) * (size_t)s->nslots)) != BFS_OK) return rc;
  s->d_slot_st = static_cast<DevState*>(p);
  if ((rc = sdalloc(s, &p, sizeof(ChunkStatus) * (size_t)s->nslots * s->ctas)) != BFS_OK) return rc;
  s->d_slot_status = static_cast<ChunkStatus*>(p);
  if ((rc = sdalloc(s, &p, sizeof(DevState))) != BFS_OK) return rc;
  s->d_st = static_cast<DevState*>(p);
  if ((rc = sdalloc(s, &p, sizeof(int32_t) * (size_t)(s->ctas + 3) / 4 * 4)) != BFS_OK) return rc;
  s->d_arrive = static_cast<int32_t*>(p);
  if ((rc = sdalloc(s, &p, sizeof(int32_t) * 4)) != BFS_OK) return rc;
  s->d_finished = static_cast<int32_t*>(p);
  if (cudaHostAlloc((void**)&s->h_slots, sizeof(SlotDev) * (size_t)s->nslots, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&s->h_st, sizeof(DevState), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return fail(BFS_E_NOMEM, "pinned host allocation failed");
  }
  int32_t* hw = nullptr;
  if (cudaHostAlloc((void**)&hw, sizeof(int32_t) * 4, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return fail(BFS_E_NOMEM, "mapped host allocation failed");
  }
  s->h_wake = hw;
  *s->h_wake = 0;
  CUDA_TRY(cudaHostGetDevicePointer((void**)&s->d_wake, hw, 0));
  memset(s->h_slots, 0, sizeof(SlotDev) * (size_t)s->nslots);
  CUDA_TRY(cudaMemsetAsync(s->d_slots, 0, sizeof(SlotDev) * (size_t)s->nslots, s->stream));
  s->running.assign((size_t)s->nslots, Query());
  s->busy.assign((size_t)s->nslots, false);
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return BFS_OK;
}

extern "C" int bfs_server_create(bfs_graph* const* graphs, int32_t ngraphs, const bfs_server_opts* opts,
                                 void* cuda_stream, bfs_server** out) {
  if (!out) return fail(BFS_E_INVAL, "out is NULL");
  *out = nullptr;
  if (!graphs || ngraphs < 1) return fail(BFS_E_INVAL, "no graphs");
  bfs_server* s = new (std::nothrow) bfs_server();
  if (!s) return fail(BFS_E_NOMEM, "host allocation failed");
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  const int rc = server_create_impl(s, graphs, ngraphs, opts);
  if (rc != BFS_OK) {
    char keep[sizeof(g_last_error)];
    memcpy(keep, g_last_error, sizeof(keep));
    bfs_server_destroy(s);
    memcpy(g_last_error, keep, sizeof(keep));
    return rc;
  }
  *out = s;
  return BFS_OK;
}

extern "C" int bfs_server_submit(bfs_server* s, int32_t graph, int32_t src, int32_t* level_out, int32_t* parent_out,
                                 int64_t tag) {
  if (!s) return fail(BFS_E_INVAL, "server is NULL");
  if (graph < 0 || graph >= (int)s->graphs.size()) return fail(BFS_E_INVAL, "graph %d out of range", graph);
  const bfs_graph* g = s->graphs[(size_t)graph];
  if (src < 0 || src >= g->n) return fail(BFS_E_INVAL, "src %d out of range [0, %d)", src, g->n);
  if (parent_out && !level_out) return fail(BFS_E_INVAL, "parent_out without level_out");
  Query q;
  q.tag = tag;
  q.graph = graph;
  q.src = src;
  q.level_out = level_out;
  q.parent_out = parent_out;
  q.lvl_dev = level_out && is_device_ptr(level_out);
  q.par_dev = parent_out && is_device_ptr(parent_out);
  q.t_submit = now_us();
  std::lock_guard<std::mutex> lock(s->mu);
  s->queue.push_back(q);
  *s->h_wake = 1;  // a running launch returns after its current step
  return BFS_OK;
}

extern "C" int bfs_server_pending(bfs_server* s, int32_t* queued, int32_t* running) {
  if (!s) return fail(BFS_E_INVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  if (queued) *queued = (int32_t)s->queue.size();
  if (running) {
    int r = 0;
    for (bool b : s->busy) r += b;
    *running = r;
  }
  return BFS_OK;
}

// Admission: the head of the queue while a slot is free and its memory fits.
static int admit(bfs_server* s) {
  while (!s->queue.empty()) {
    int slot = -1;
    for (int i = 0; i < s->nslots; ++i)
      if (!s->busy[(size_t)i]) {
        slot = i;
        break;
      }
    if (slot < 0) return BFS_OK;
    Query q = s->queue.front();
    bfs_graph* g = s->graphs[(size_t)q.graph];
    const bool in_place = q.lvl_dev && !g->relabel;  // kernels write the caller's device buffers
    const bool internal = !in_place || (q.parent_out && !q.par_dev);
    const bool stage = g->relabel && q.level_out && (!q.lvl_dev || (q.parent_out && !q.par_dev));
    const size_t need = query_bytes(g, true, stage);
    size_t off = 0;
    if (!s->arena.alloc(need, &off)) {
      if (need > s->arena.bytes) {
        s->queue.pop_front();
        bfs_completion c;
        memset(&c, 0, sizeof(c));
        c.tag = q.tag;
        c.graph = q.graph;
        c.src = q.src;
        c.status = BFS_E_NOMEM;
        c.t_submit_us = q.t_submit;
        c.t_done_us = now_us();
        s->done.push_back(c);
        continue;
      }
      return BFS_OK;  // wait until running queries free memory
    }
    (void)internal;
    s->queue.pop_front();
    q.arena_off = off;
    q.arena_bytes = need;
    char* cur = s->arena.base + off;
    auto take = [&](size_t bytes) {
      char* r = cur;
      cur += align256(bytes);
      return r;
    };
    const size_t n = (size_t)g->n, m = (size_t)g->nnz;
    Params p;
    memset(&p, 0, sizeof(p));
    p.n = g->n;
    p.nnz = g->nnz;
    p.row_ptr = g->d_row_ptr;
    p.col_idx = g->d_col_idx;
    for (int b = 0; b < 2; ++b) {
      p.F[b] = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (n + 4)));
      p.RS[b] = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (n + 4)));
      p.EX[b] = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (n + 4)));
    }
    p.cand = reinterpret_cast<int2*>(take(sizeof(int2) * (m + 32)));
    p.cand_aux = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (m + 32)));
    int32_t* lv_int = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (n + 4)));
    int32_t* pa_int = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (n + 4)));
    q.stage = stage ? reinterpret_cast<int32_t*>(take(2 * sizeof(int32_t) * (n + 4))) : nullptr;
    q.level = in_place ? q.level_out : lv_int;
    q.parent = (in_place && q.par_dev) ? q.parent_out : pa_int;
    p.level = q.level;
    p.parent = q.parent;
    p.cand_cnt = nullptr;
    p.status = s->d_slot_status + (size_t)slot * s->ctas;
    p.bar_arrive = nullptr;
    p.cta_smid = nullptr;
    p.st = s->d_slot_st + slot;
    p.lvl = nullptr;
    p.lvl_cap = 0;
    p.grain = s->grain;
    p.work_insensitive = 0;
    p.src = g->relabel ? g->h_inv[(size_t)q.src] : q.src;
    p.guess_search = g->relabel ? 0 : 1;
    p.max_chunks = s->ctas;
    p.debug_flags = 0;
    p.spin_ns = s->spin_ns;
    p.hub_bits = nullptr;
    p.hub_n = 0;
    p.small_edges = 0;
    SlotDev& sd = s->h_slots[slot];
    memset(&sd, 0, sizeof(sd));
    sd.p = p;
    sd.level = 0;
    sd.active = 1;
    CUDA_TRY(cudaMemcpyAsync(s->d_slots + slot, &sd, sizeof(SlotDev), cudaMemcpyHostToDevice, s->stream));
    const int grid = std::max(1, std::min(s->sms * 8, (int)((n / 4 + 255) / 256)));
    k_serve_init<<<grid, 256, 0, s->stream>>>(p, s->d_slots + slot);
    CUDA_TRY(cudaGetLastError());
    q.t_admit = now_us();
    s->running[(size_t)slot] = q;
    s->busy[(size_t)slot] = true;
  }
  return BFS_OK;
}

// Outputs of a finished query where the caller wants them; frees its memory.
static int retire(bfs_server* s, int slot, int status, bfs_completion* c) {
  Query& q = s->running[(size_t)slot];
  const bfs_graph* g = s->graphs[(size_t)q.graph];
  const SlotDev& sd = s->h_slots[slot];
  const size_t n = (size_t)g->n;
  if (status == BFS_OK && q.level_out) {
    if (g->relabel) {
      int32_t* lo = q.lvl_dev ? q.level_out : q.stage;
      int32_t* po = q.parent_out ? (q.par_dev ? q.parent_out : q.stage + n + 4) : nullptr;
      const int grid = std::max(1, std::min(s->sms * 8, (int)((n + 255) / 256)));
      k_serve_finalize<<<grid, 256, 0, s->stream>>>(g->n, g->d_inv, g->d_perm, q.level, q.parent, lo, po);
      CUDA_TRY(cudaGetLastError());
      if (!q.lvl_dev)
        CUDA_TRY(cudaMemcpyAsync(q.level_out, lo, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->stream));
      if (q.parent_out && !q.par_dev)
        CUDA_TRY(cudaMemcpyAsync(q.parent_out, po, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->stream));
    } else {
      if (!q.lvl_dev)
        CUDA_TRY(cudaMemcpyAsync(q.level_out, q.level, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->stream));
      if (q.parent_out && q.parent != q.parent_out)
        CUDA_TRY(cudaMemcpyAsync(q.parent_out, q.parent, sizeof(int32_t) * n, cudaMemcpyDefault, s->stream));
    }
  }
  memset(c, 0, sizeof(*c));
  c->tag = q.tag;
  c->graph = q.graph;
  c->src = q.src;
  c->status = status;
  c->num_levels = sd.num_levels;
  c->reached = sd.reached;
  c->edges_scanned = sd.edges;
  c->t_submit_us = q.t_submit;
  c->t_admit_us = q.t_admit;
  s->arena.release(q.arena_off, q.arena_bytes);
  s->busy[(size_t)slot] = false;
  return BFS_OK;
}

// One scheduling round.  Called with s->mu held; the lock is released while
// the launch runs on the GPU, so that other threads can submit meanwhile (a
// submission sets the wake flag and the launch returns after its step).
static int poll_impl(bfs_server* s, std::unique_lock<std::mutex>& lock) {
  int rc = admit(s);
  if (rc != BFS_OK) return rc;
  bool any = false;
  for (bool b : s->busy) any |= b;
  if (!any) return BFS_OK;
  // one launch over all running queries
  ServeParams sp;
  memset(&sp, 0, sizeof(sp));
  sp.slots = s->d_slots;
  sp.nslots = s->nslots;
  sp.max_levels = s->levels_per_launch;
  sp.grain = s->grain;
  sp.local_levels = s->local_levels;
  sp.local_edges = 256 * s->wpc;
  sp.finished = s->d_finished;
  sp.wake = s->d_wake;
  sp.st = s->d_st;
  sp.bar_arrive = s->d_arrive;
  sp.spin_ns = s->spin_ns;
  sp.debug_flags = 0;
  // submissions from now on end the launch early; the queries still queued
  // (no slot or no memory) wait for a query to finish, which ends it anyway
  *s->h_wake = 0;
  CUDA_TRY(cudaMemsetAsync(s->d_st, 0, sizeof(DevState), s->stream));
  CUDA_TRY(cudaMemsetAsync(s->d_arrive, 0, sizeof(int32_t) * ((size_t)(s->ctas + 3) / 4 * 4), s->stream));
  CUDA_TRY(cudaMemsetAsync(s->d_finished, 0, sizeof(int32_t), s->stream));
  void* args[] = {&sp};
  const void* fn = serve_fn(s->wpc);
  CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(s->ctas), dim3(s->wpc * kWarp), args, 0, s->stream));
  CUDA_TRY(cudaMemcpyAsync(s->h_slots, s->d_slots, sizeof(SlotDev) * (size_t)s->nslots, cudaMemcpyDeviceToHost,
                           s->stream));
  CUDA_TRY(cudaMemcpyAsync(s->h_st, s->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
  lock.unlock();
  const cudaError_t sync_err = cudaStreamSynchronize(s->stream);
  lock.lock();
  CUDA_TRY(sync_err);
  const int server_err = s->h_st->err;
  std::vector<bfs_completion> fin;
  for (int i = 0; i < s->nslots; ++i) {
    if (!s->busy[(size_t)i]) continue;
    const SlotDev& sd = s->h_slots[i];
    if (sd.active && !server_err) continue;
    DevState qst;
    CUDA_TRY(cudaMemcpyAsync(&qst, s->d_slot_st + i, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    const int status = server_err ? server_err : qst.err;
    bfs_completion c;
    if ((rc = retire(s, i, status, &c)) != BFS_OK) return rc;
    fin.push_back(c);
  }
  if (server_err) {
    // a device wait ran out: every running query was failed above
    CUDA_TRY(cudaMemsetAsync(s->d_slots, 0, sizeof(SlotDev) * (size_t)s->nslots, s->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));  // outputs are in place
  const double t = now_us();
  for (auto& c : fin) {
    c.t_done_us = t;
    s->done.push_back(c);
  }
  return BFS_OK;
}

extern "C" int bfs_server_poll(bfs_server* s, bfs_completion* out, int32_t cap, int32_t* ndone) {
  if (!s) return fail(BFS_E_INVAL, "server is NULL");
  if (ndone) *ndone = 0;
  std::unique_lock<std::mutex> lock(s->mu);
  if (s->polling) return fail(BFS_E_INVAL, "bfs_server_poll called from two threads at once");
  s->polling = true;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    s->polling = false;
    return fail(BFS_E_CUDA, "cudaGetDevice failed");
  }
  if (cur != s->device) cudaSetDevice(s->device);
  const int rc = poll_impl(s, lock);
  if (cur != s->device) cudaSetDevice(cur);
  s->polling = false;
  int k = 0;
  while (out && k < cap && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  if (ndone) *ndone = k;
  return rc;
}
