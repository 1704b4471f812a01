// S3BFS level-step library for GB300 (sm_103a): kernels and the C ABI.
//
// Public interface: include/s3bfs.h.  Kernels: level_loop.cuh (level loop),
// msbfs.cuh (bitmask batches); their device building blocks:
// s3bfs_device.cuh.  Host-side CSR checks: csr_host.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "host_internal.h"
#include "msbfs.cuh"
#include "level_loop.cuh"
#include "s3bfs.h"
#include "s3bfs_device.cuh"

using namespace s3bfs;

// host-side CSR helpers (csr_host.cpp)
int s3bfs_host_check_duplicates(int32_t n, const int32_t* rp, const int32_t* ci, char* msg, size_t len);
int s3bfs_host_dedup(int32_t n, const int32_t* rp, const int32_t* ci, std::vector<int32_t>* rp_out,
                     std::vector<int32_t>* ci_out);
double s3bfs_host_top_degree_share(int32_t n, const int32_t* rp, int32_t top);
int s3bfs_host_is_symmetric(int32_t n, const int32_t* rp, const int32_t* ci);
int s3bfs_host_relabel(int32_t n, const int32_t* rp, const int32_t* ci, bool sort_rows, std::vector<int32_t>* perm,
                       std::vector<int32_t>* inv, std::vector<int32_t>* rp_out, std::vector<int32_t>* ci_out);

// dynamic shared memory of the level loop: the visited bits
static size_t loop_smem(int hub_n) { return (size_t)hub_n / 8; }

// A graph that is not renumbered gets a visited bit for every vertex up to
// this size (128 KB of shared memory) when its traversals are top-down only.
// Bottom-up levels test level[] through L1, which the larger bitmap would
// shrink, so with them the limit stays kHubMax.
constexpr int kBitsAllMax = 1 << 20;

// the level loop for a CTA shape; DO: with bottom-up levels (a separate
// kernel, so that the top-down loop carries no trace of them)
static const void* level_loop_fn(int wpc, bool DO) {
  switch (wpc) {
    case 32: return DO ? (const void*)k_level_loop<32, true> : (const void*)k_level_loop<32, false>;
    case 24: return DO ? (const void*)k_level_loop<24, true> : (const void*)k_level_loop<24, false>;
    case 16: return DO ? (const void*)k_level_loop<16, true> : (const void*)k_level_loop<16, false>;
    default: return DO ? (const void*)k_level_loop<8, true> : (const void*)k_level_loop<8, false>;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

thread_local char g_last_error[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" const char* bfs_strerror(int code) {
  switch (code) {
    case BFS_OK: return "ok";
    case BFS_E_INVAL: return "invalid argument";
    case BFS_E_MULTIGRAPH: return "repeated neighbour in a CSR row (the graph must be simple)";
    case BFS_E_NOMEM: return "out of memory";
    case BFS_E_CUDA: return "CUDA error";
    case BFS_E_TIMEOUT: return "device wait timed out";
    case BFS_E_CHECK: return "index out of range (checked build)";
    default: return "unknown error";
  }
}

extern "C" const char* bfs_last_error(void) { return g_last_error; }

extern "C" void bfs_destroy(bfs_graph* g) {
  if (!g) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (void* p : g->allocs) cudaFree(p);
  if (g->h_st) cudaFreeHost(g->h_st);
  if (g->h_smid) cudaFreeHost(g->h_smid);
  if (g->h_ctrl) cudaFreeHost(g->h_ctrl);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  if (g->copy_stream) {
    cudaStreamSynchronize(g->copy_stream);
    cudaStreamDestroy(g->copy_stream);
  }
  for (int s = 0; s < bfs_graph::kQueueDepth; ++s) {
    for (auto& e : g->slot_ev[s])
      if (e) cudaEventDestroy(e);
    if (g->slot_ready[s]) cudaEventDestroy(g->slot_ready[s]);
    if (g->slot_copied[s]) cudaEventDestroy(g->slot_copied[s]);
  }
  if (g->h_slot_st) cudaFreeHost(g->h_slot_st);
  cudaSetDevice(cur);
  delete g;
}

extern "C" int64_t bfs_graph_device_bytes(const bfs_graph* g) { return g ? (int64_t)g->dev_bytes : -1; }

extern "C" int bfs_graph_info(const bfs_graph* g, int32_t* n, int32_t* nnz, int32_t* ctas, int32_t* warps) {
  if (!g) return fail(BFS_E_INVAL, "graph is NULL");
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (ctas) *ctas = g->ctas;
  if (warps) *warps = g->warps;
  return BFS_OK;
}

static int create_impl(bfs_graph* g, int32_t n, int32_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                       int flags, const bfs_opts* opts) {
  int rc;
  CUDA_TRY(cudaGetDevice(&g->device));
  CUDA_TRY(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device));
  int coop = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device));
  if (opts) {
    if (opts->chunk_edges > 0) g->grain = opts->chunk_edges;
    if (opts->reserved != 0) return fail(BFS_E_INVAL, "bfs_opts.reserved must be 0");
    if (opts->max_device_bytes < 0) return fail(BFS_E_INVAL, "max_device_bytes must be >= 0");
    g->dev_cap = (size_t)opts->max_device_bytes;
    if (opts->persistent < 0) g->persistent = 0;
    g->work_insensitive = opts->work_insensitive != 0;
    if (opts->spin_limit_ms > 0) g->spin_ns = (long long)opts->spin_limit_ms * 1000000ll;
    g->debug_flags = opts->debug_flags;
    g->batch_bitmask = opts->batch_bitmask;
    if (opts->small_level_edges > 0) g->small_edges = opts->small_level_edges;
    if (opts->small_level_edges < 0) g->small_edges = 0;  // never
    if (opts->direction != 0 && opts->direction != 1)
      return fail(BFS_E_INVAL, "direction = %d: use 0 or 1", opts->direction);
    g->direction = opts->direction;
    if (opts->do_alpha < 0 || opts->do_beta < 0) return fail(BFS_E_INVAL, "do_alpha / do_beta must be >= 0");
    if (opts->do_alpha > 0) g->alpha = opts->do_alpha;
    if (opts->do_beta > 0) g->beta = opts->do_beta;
    if (opts->do_gamma < -1) return fail(BFS_E_INVAL, "do_gamma = %d: use -1 (off), 0 (default) or > 0", opts->do_gamma);
    if (opts->do_gamma > 0) g->gamma = opts->do_gamma;
    if (opts->do_gamma == -1) g->gamma = 0;
  }
  if (g->direction && !(flags & BFS_SYMMETRIC))
    return fail(BFS_E_INVAL, "direction-optimising levels need a symmetric graph (BFS_SYMMETRIC)");
  g->symmetric = (flags & BFS_SYMMETRIC) != 0;
  if (!coop) g->persistent = 0;

  // CSR: host data is validated / cleaned on the host, then uploaded
  std::vector<int32_t> h_rp, h_ci;
  const bool dev_in = (flags & BFS_DEVICE_PTRS) != 0;
  const int32_t* rp = row_ptr;
  const int32_t* ci = col_idx;
  if (flags & (BFS_VALIDATE | BFS_DEDUP)) {
    if (dev_in) {
      h_rp.resize((size_t)n + 1);
      CUDA_TRY(cudaMemcpy(h_rp.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost));
      if (h_rp[n] != nnz || h_rp[0] != 0) return fail(BFS_E_INVAL, "row_ptr[0] must be 0 and row_ptr[n] == nnz");
      h_ci.resize((size_t)std::max(nnz, 1));
      if (nnz) CUDA_TRY(cudaMemcpy(h_ci.data(), col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost));
      rp = h_rp.data();
      ci = h_ci.data();
    }
    if (rp[0] != 0 || rp[n] != nnz) return fail(BFS_E_INVAL, "row_ptr[0] must be 0 and row_ptr[n] == nnz");
    for (int32_t v = 0; v < n; ++v)
      if (rp[v] > rp[v + 1]) return fail(BFS_E_INVAL, "row_ptr decreases at %d", v);
    for (int32_t e = 0; e < nnz; ++e)
      if (ci[e] < 0 || ci[e] >= n) return fail(BFS_E_INVAL, "col_idx[%d] = %d out of range", e, ci[e]);
    if (flags & BFS_DEDUP) {
      std::vector<int32_t> rp2, ci2;
      if (s3bfs_host_dedup(n, rp, ci, &rp2, &ci2) != 0) return fail(BFS_E_NOMEM, "dedup: host allocation failed");
      h_rp.swap(rp2);
      h_ci.swap(ci2);
      rp = h_rp.data();
      ci = h_ci.data();
      nnz = h_rp[n];
    } else {
      char msg[256];
      if (s3bfs_host_check_duplicates(n, rp, ci, msg, sizeof(msg)) != 0) return fail(BFS_E_MULTIGRAPH, "%s", msg);
    }
    if ((flags & BFS_SYMMETRIC) && !s3bfs_host_is_symmetric(n, rp, ci))
      return fail(BFS_E_INVAL, "BFS_SYMMETRIC: an edge lacks its reverse");
  }
  // shared-memory visited bits: every vertex when n is small (kHubMax; up to
  // kBitsAllMax for a graph that is not skewed, top-down only), else the
  // kHubMax highest-degree vertices after a degree-descending renumbering,
  // if they hold at least half of the edge endpoints (skewed graphs)
  bool csr_on_host = !dev_in || !h_rp.empty();  // rp / ci are host arrays
  const int relabel_opt = opts ? opts->relabel : 0;
  if (relabel_opt >= 0) {
    if (n <= kHubMax && relabel_opt == 0) {
      g->hub_n = (n + 127) / 128 * 128;
    } else {
      std::vector<int32_t> rp_probe;
      const int32_t* rpp = rp;
      if (!csr_on_host) {
        rp_probe.resize((size_t)n + 1);
        CUDA_TRY(cudaMemcpy(rp_probe.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost));
        rpp = rp_probe.data();
      }
      if (rpp[0] != 0 || rpp[n] != nnz) return fail(BFS_E_INVAL, "row_ptr[0] must be 0 and row_ptr[n] == nnz");
      for (int32_t v = 0; v < n; ++v)
        if (rpp[v] > rpp[v + 1]) return fail(BFS_E_INVAL, "row_ptr decreases at %d", v);
      const bool skewed = s3bfs_host_top_degree_share(n, rpp, kHubMax) >= 0.5;
      if (relabel_opt == 1 || skewed) {
        if (!csr_on_host) {
          h_rp.swap(rp_probe);
          h_ci.resize((size_t)std::max(nnz, 1));
          if (nnz)
            CUDA_TRY(cudaMemcpy(h_ci.data(), col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost));
          rp = h_rp.data();
          ci = h_ci.data();
          csr_on_host = true;
        }
        for (int32_t e = 0; e < nnz; ++e)
          if (ci[e] < 0 || ci[e] >= n) return fail(BFS_E_INVAL, "col_idx[%d] = %d out of range", e, ci[e]);
        std::vector<int32_t> perm, rp2, ci2;
        if (s3bfs_host_relabel(n, rp, ci, g->direction != 0, &perm, &g->h_inv, &rp2, &ci2) != 0)
          return fail(BFS_E_NOMEM, "renumbering: host allocation failed");
        h_rp.swap(rp2);
        h_ci.swap(ci2);
        rp = h_rp.data();
        ci = h_ci.data();
        g->relabel = true;
        g->hub_n = std::min(kHubMax, (n + 127) / 128 * 128);
        if ((rc = dalloc(g, &g->d_perm, (size_t)n)) != BFS_OK) return rc;
        if ((rc = dalloc(g, &g->d_inv, (size_t)n)) != BFS_OK) return rc;
        CUDA_TRY(cudaMemcpyAsync(g->d_perm, perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                                 g->stream));
        CUDA_TRY(cudaMemcpyAsync(g->d_inv, g->h_inv.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                                 g->stream));
        CUDA_TRY(cudaStreamSynchronize(g->stream));
      } else if (relabel_opt == 0 && !g->direction && n <= kBitsAllMax) {
        g->hub_n = (n + 127) / 128 * 128;
      }
    }
  }
  const bool upload_from_host = csr_on_host;
  if (g->direction || g->symmetric) {
    // vertices of degree > 0: the ones a bottom-up level can find (and, on a
    // symmetric graph, the count that decides how a bitmask batch writes -1)
    std::vector<int32_t> rp_copy;
    const int32_t* rpp = rp;
    if (!csr_on_host) {
      rp_copy.resize((size_t)n + 1);
      CUDA_TRY(cudaMemcpy(rp_copy.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost));
      rpp = rp_copy.data();
    }
    int32_t live = 0;
    for (int32_t v = 0; v < n; ++v) live += rpp[v + 1] > rpp[v];
    g->n_live = live;
  }
  g->n = n;
  g->nnz = nnz;
  const size_t nnz_pad = ((size_t)nnz + 3) / 4 * 4 + 4;
  if ((rc = dalloc(g, &g->d_row_ptr, (size_t)n + 1)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_col_idx, nnz_pad)) != BFS_OK) return rc;
  const cudaMemcpyKind kind = upload_from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CUDA_TRY(cudaMemcpyAsync(g->d_row_ptr, rp, sizeof(int32_t) * ((size_t)n + 1), kind, g->stream));
  CUDA_TRY(cudaMemsetAsync(g->d_col_idx, 0, sizeof(int32_t) * nnz_pad, g->stream));
  if (nnz) CUDA_TRY(cudaMemcpyAsync(g->d_col_idx, ci, sizeof(int32_t) * (size_t)nnz, kind, g->stream));

  // CTA shape: one CTA of 32 warps per SM when the visited bits are in shared
  // memory (one copy per SM), else one 16-warp CTA per SM (128 registers a
  // thread, no spills, half the CTAs at every grid barrier): the graphs
  // without visited bits are the large flat ones, whose thousands of small
  // levels are bound by per-level latency (grid 4096^2: 81.7 against 112.4 ms
  // per traversal with 8-warp CTAs, same box)
  const int cw = opts ? opts->cta_warps : 0;
  if (cw != 0 && cw != 8 && cw != 16 && cw != 24 && cw != 32)
    return fail(BFS_E_INVAL, "cta_warps = %d: use 0, 8, 16, 24 or 32", cw);
  g->wpc = cw ? cw : (g->hub_n > 0 ? 32 : 16);
  // persistent grid: every CTA that fits next to the shared-memory bits
  const void* loop_fn = level_loop_fn(g->wpc, g->direction != 0);
  // the attribute is per kernel, shared by every graph: set it to the largest size any graph uses
  CUDA_TRY(cudaFuncSetAttribute(loop_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)loop_smem(std::max(kHubMax, kBitsAllMax))));
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, loop_fn, g->wpc * kWarp, loop_smem(g->hub_n)));
  if (per_sm < 1) return fail(BFS_E_CUDA, "level-loop kernel cannot be resident (occupancy 0)");
  g->ctas = per_sm * g->sms;
  if (opts && opts->ctas > 0) g->ctas = std::min(g->ctas, (int)opts->ctas);
  g->warps = g->ctas * g->wpc;
  if (g->small_edges < 0) g->small_edges = 256 * g->wpc;
  // the work-insensitive comparison arm runs every level on every warp of the grid
  if (g->work_insensitive) g->small_edges = 0;

  // work memory
  if (g->hub_n > 0 && (rc = dalloc(g, &g->d_hub_bits, (size_t)g->hub_n / 32)) != BFS_OK) return rc;
  if (g->relabel) {
    if ((rc = dalloc(g, &g->d_out_level, (size_t)n)) != BFS_OK) return rc;
    if ((rc = dalloc(g, &g->d_out_parent, (size_t)n)) != BFS_OK) return rc;
  }
  g->lvl_cap = (int32_t)std::min<long long>((long long)n + 1, 1 << 20);
  const int max_chunks = g->warps;
  if ((rc = dalloc(g, &g->d_level, (size_t)n + 4)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_parent, (size_t)n + 4)) != BFS_OK) return rc;
  for (int b = 0; b < 2; ++b) {
    if ((rc = dalloc(g, &g->d_F[b], (size_t)n + 4)) != BFS_OK) return rc;
    if ((rc = dalloc(g, &g->d_RS[b], (size_t)n + 4)) != BFS_OK) return rc;
    if ((rc = dalloc(g, &g->d_EX[b], (size_t)n + 4)) != BFS_OK) return rc;
  }
  // candidates: one slot per edge of a top-down level; a bottom-up level
  // gives each warp room for the 128 vertices of each group of four bitmap
  // words it owns
  size_t cand_cap = (size_t)nnz + 32;
  if (g->direction) {
    g->nwords = (int32_t)(((long long)n + 127) / 128 * 4);
    const size_t gpw = ((size_t)g->nwords / 4 + g->warps - 1) / g->warps;
    cand_cap = std::max(cand_cap, gpw * 128 * (size_t)g->warps + 32);
    for (int b = 0; b < 2; ++b)
      if ((rc = dalloc(g, &g->d_fb[b], (size_t)g->nwords)) != BFS_OK) return rc;
    if ((rc = dalloc(g, &g->d_ulist, cand_cap)) != BFS_OK) return rc;
    if ((rc = dalloc(g, &g->d_ulist_cnt, (size_t)g->warps)) != BFS_OK) return rc;
  }
  if ((rc = dalloc(g, &g->d_cand, cand_cap)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_cand_aux, cand_cap)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_cand_cnt, (size_t)max_chunks)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_status, (size_t)max_chunks)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_arrive, (size_t)(g->ctas + 3) / 4 * 4)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_smid, (size_t)g->ctas)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_st, 1)) != BFS_OK) return rc;
  if ((rc = dalloc(g, &g->d_lvl, (size_t)g->lvl_cap * kLevelFields)) != BFS_OK) return rc;
  CUDA_TRY(cudaMemsetAsync(g->d_status, 0, sizeof(ChunkStatus) * (size_t)max_chunks, g->stream));
  CUDA_TRY(cudaMemsetAsync(g->d_st, 0, sizeof(DevState), g->stream));
  if (cudaHostAlloc((void**)&g->h_st, sizeof(DevState), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void**)&g->h_smid, sizeof(int32_t) * (size_t)g->ctas, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&g->h_ctrl, sizeof(LevelCtrl) * 2 + 16, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return fail(BFS_E_NOMEM, "pinned host allocation failed");
  }
  // k_finalize writes a renumbered graph's state block through the device's
  // view of h_st; without one it is copied after the kernel instead
  if (cudaHostGetDevicePointer((void**)&g->h_st_map, g->h_st, 0) != cudaSuccess) {
    cudaGetLastError();
    g->h_st_map = nullptr;
  }
  for (auto& e : g->ev) CUDA_TRY(cudaEventCreate(&e));

  // device-side range checks (always: they guard every later access)
  int* d_bad = nullptr;
  if ((rc = dalloc(g, &d_bad, 1)) != BFS_OK) return rc;
  CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), g->stream));
  const int cgrid = std::max(1, std::min(g->sms * 8, (int)(((long long)std::max(n, nnz) + 255) / 256)));
  k_check_csr<<<cgrid, 256, 0, g->stream>>>(n, nnz, g->d_row_ptr, g->d_col_idx, d_bad);
  CUDA_TRY(cudaGetLastError());
  int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (bad == 1) return fail(BFS_E_INVAL, "row_ptr must start at 0, never decrease and end at nnz");
  if (bad == 2) return fail(BFS_E_INVAL, "col_idx entry out of range [0, n)");
  return BFS_OK;
}

extern "C" int bfs_create_csr(int32_t n, int32_t nnz, const int32_t* row_ptr, const int32_t* col_idx, int flags,
                              const bfs_opts* opts, void* cuda_stream, bfs_graph** out) {
  if (!out) return fail(BFS_E_INVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 0x7FFFFFFF - 8) return fail(BFS_E_INVAL, "n = %d out of range [1, 2^31-8)", n);
  if (nnz < 0 || nnz > 0x7FFFFFFF - 64) return fail(BFS_E_INVAL, "nnz = %d out of range", nnz);
  if (!row_ptr || (nnz > 0 && !col_idx)) return fail(BFS_E_INVAL, "NULL CSR array");
  if (flags & ~(BFS_DEVICE_PTRS | BFS_VALIDATE | BFS_DEDUP | BFS_SYMMETRIC))
    return fail(BFS_E_INVAL, "unknown flags 0x%x", flags);
  bfs_graph* g = new (std::nothrow) bfs_graph();
  if (!g) return fail(BFS_E_NOMEM, "host allocation failed");
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  const int rc = create_impl(g, n, nnz, row_ptr, col_idx, flags, opts);
  if (rc != BFS_OK) {
    char keep[sizeof(g_last_error)];
    memcpy(keep, g_last_error, sizeof(keep));
    bfs_destroy(g);
    memcpy(g_last_error, keep, sizeof(keep));
    return rc;
  }
  *out = g;
  return BFS_OK;
}

static Params make_params(bfs_graph* g, int32_t src, int32_t* level, int32_t* parent) {
  Params p;
  memset(&p, 0, sizeof(p));
  p.n = g->n;
  p.nnz = g->nnz;
  p.row_ptr = g->d_row_ptr;
  p.col_idx = g->d_col_idx;
  p.level = level;
  p.parent = parent;
  // a renumbered graph's outputs always pass through k_finalize
  p.parent_lazy = g->relabel ? 1 : 0;
  // graphs renumbered by degree are the skewed ones, where a proportional
  // guess of the start entry misses
  p.guess_search = g->relabel ? 0 : 1;
  for (int b = 0; b < 2; ++b) {
    p.F[b] = g->d_F[b];
    p.RS[b] = g->d_RS[b];
    p.EX[b] = g->d_EX[b];
  }
  p.cand = g->d_cand;
  p.cand_aux = g->d_cand_aux;
  p.cand_cnt = g->d_cand_cnt;
  p.status = g->d_status;
  p.bar_arrive = g->d_arrive;
  p.cta_smid = g->d_smid;
  p.st = g->d_st;
  p.lvl = g->d_lvl;
  p.lvl_cap = g->lvl_cap;
  p.grain = g->grain;
  p.work_insensitive = g->work_insensitive;
  p.src = src;
  p.max_chunks = g->warps;
  p.debug_flags = g->debug_flags;
  p.spin_ns = g->spin_ns;
  p.hub_bits = g->d_hub_bits;
  p.hub_n = g->persistent ? g->hub_n : 0;
  p.small_edges = g->persistent ? g->small_edges : 0;
  p.fb[0] = g->d_fb[0];
  p.fb[1] = g->d_fb[1];
  p.nwords = g->nwords;
  // degree-descending renumbering puts the vertices of degree 0 last; on a
  // symmetric graph those are the n - n_live isolated ones, which no level
  // reaches (on a directed one a vertex without out-edges may be reached)
  const bool isolated_last = g->relabel && g->symmetric && g->n_live > 0;
  p.bu_groups = isolated_last ? (int32_t)(((long long)g->n_live + 127) / 128) : g->nwords / 4;
  p.level_n = isolated_last ? g->n_live : g->n;
  p.ulist = g->d_ulist;
  p.ulist_cnt = g->d_ulist_cnt;
  p.direction = g->persistent ? g->direction : 0;
  p.alpha = g->alpha;
  p.beta = g->beta;
  p.gamma = g->gamma;
  p.n_live = g->n_live;
#if S3BFS_CHECKED
  p.fdump = g->fdump_on ? g->d_fdump : nullptr;
#endif
  return p;
}

// Enqueue one traversal (init + level loop) on the graph's stream.
// ev: three events recorded before init, before the level loop and after it
// (null: untimed)
static int enqueue_traversal(bfs_graph* g, const Params& p, cudaEvent_t* ev) {
  const bool timed = ev != nullptr;
  if (timed) CUDA_TRY(cudaEventRecord(ev[0], g->stream));
  // one 1024-thread block per SM (k_init holds the whole parameter block in
  // registers, so a second one does not fit), grid-stride over the arrays
  const int igrid = std::max(1, std::min(g->sms, (int)(((long long)g->n / 4 + kThreads - 1) / kThreads)));
  k_init<<<igrid, kThreads, 0, g->stream>>>(p, g->ctas);
  CUDA_TRY(cudaGetLastError());
  ++g->launches;
  if (timed) CUDA_TRY(cudaEventRecord(ev[1], g->stream));
  if (g->persistent) {
    Params pc = p;
    void* args[] = {&pc};
    CUDA_TRY(cudaLaunchCooperativeKernel(level_loop_fn(g->wpc, p.direction != 0), dim3(g->ctas),
                                         dim3(g->wpc * kWarp), args,
                                         loop_smem(p.hub_n), g->stream));
    ++g->launches;
  } else {
    // launch per phase; the host reads n and e of every level
    LevelCtrl* hc = reinterpret_cast<LevelCtrl*>(g->h_ctrl);
    int l = 0;
    CUDA_TRY(cudaMemcpyAsync(hc, &g->d_st->ctrl[0], sizeof(LevelCtrl), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    long long reached = 0, edges = 0, cands = 0;
    while (hc->n > 0) {
      const int n_l = hc->n, e_l = hc->e;
      int P_l, C_l;
      level_sizing(e_l, g->warps, g->grain, g->work_insensitive, &P_l, &C_l);
      reached += n_l;
      edges += e_l;
      const int grid = std::max(1, (P_l + g->wpc - 1) / g->wpc);
      switch (g->wpc) {
        case 32:
          k_explore<32><<<grid, 32 * kWarp, 0, g->stream>>>(p, l, n_l, e_l, P_l, C_l);
          k_compact<32><<<grid, 32 * kWarp, 0, g->stream>>>(p, l, e_l, P_l, C_l);
          break;
        case 24:
          k_explore<24><<<grid, 24 * kWarp, 0, g->stream>>>(p, l, n_l, e_l, P_l, C_l);
          k_compact<24><<<grid, 24 * kWarp, 0, g->stream>>>(p, l, e_l, P_l, C_l);
          break;
        case 16:
          k_explore<16><<<grid, 16 * kWarp, 0, g->stream>>>(p, l, n_l, e_l, P_l, C_l);
          k_compact<16><<<grid, 16 * kWarp, 0, g->stream>>>(p, l, e_l, P_l, C_l);
          break;
        default:
          k_explore<8><<<grid, 8 * kWarp, 0, g->stream>>>(p, l, n_l, e_l, P_l, C_l);
          k_compact<8><<<grid, 8 * kWarp, 0, g->stream>>>(p, l, e_l, P_l, C_l);
      }
      CUDA_TRY(cudaGetLastError());
      g->launches += 2;
      CUDA_TRY(cudaMemcpyAsync(hc, &g->d_st->ctrl[(l + 1) & 1], sizeof(LevelCtrl), cudaMemcpyDeviceToHost,
                               g->stream));
      CUDA_TRY(cudaMemcpyAsync(hc + 1, &g->d_st->err, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
      CUDA_TRY(cudaStreamSynchronize(g->stream));
      if (reinterpret_cast<int32_t*>(hc + 1)[0] != 0) break;
      cands += hc->c;
      ++l;
    }
    DevState tail;
    memset(&tail, 0, sizeof(tail));
    tail.num_levels = l;
    tail.reached = reached;
    tail.edges = edges;
    tail.cands = cands;
    tail.work = edges;
    // num_levels and totals go to the device block so both modes read back alike
    CUDA_TRY(cudaMemcpyAsync(&g->d_st->num_levels, &tail.num_levels, sizeof(int32_t), cudaMemcpyHostToDevice,
                             g->stream));
    CUDA_TRY(cudaMemcpyAsync(&g->d_st->reached, &tail.reached, 3 * sizeof(long long), cudaMemcpyHostToDevice,
                             g->stream));
    CUDA_TRY(cudaMemcpyAsync(&g->d_st->work, &tail.work, sizeof(long long), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
  }
  CUDA_TRY(cudaGetLastError());
  if (timed) CUDA_TRY(cudaEventRecord(ev[2], g->stream));
  return BFS_OK;
}

// The traversal's outcome from its device state block (copied to the host).
static int traversal_error(const DevState& st, int32_t src) {
  if (st.err == 0) return BFS_OK;
  if (st.err == BFS_E_TIMEOUT) return fail(BFS_E_TIMEOUT, "device wait %d ran out (src %d)", st.err_where, src);
  if (st.err == BFS_E_MULTIGRAPH)
    return fail(BFS_E_MULTIGRAPH, "next frontier larger than n: the graph repeats a neighbour (src %d)", src);
  if (st.err == BFS_E_CHECK) return fail(BFS_E_CHECK, "range check %d failed (src %d)", st.err_where, src);
  return fail(st.err, "device error %d at %d (src %d)", st.err, st.err_where, src);
}

// Totals and times of a finished traversal (ev: its three events, or null).
static int traversal_stats(const bfs_graph* g, const DevState& st, int launches, cudaEvent_t* ev, bfs_stats* stats) {
  stats->num_levels = st.num_levels;
  stats->active_ctas = g->persistent ? g->ctas : 0;
  stats->reached = st.reached;
  stats->edges_scanned = st.edges;
  stats->candidates = st.cands;
  stats->ms_level_step = 0.f;
  stats->ms_total = 0.f;
  stats->work_edges = st.work;
  stats->launches = launches;
  if (ev) {
    CUDA_TRY(cudaEventElapsedTime(&stats->ms_level_step, ev[1], ev[2]));
    CUDA_TRY(cudaEventElapsedTime(&stats->ms_total, ev[0], ev[2]));
  }
  return BFS_OK;
}

// state_on_host: k_finalize already wrote the state block into h_st
static int finish_traversal(bfs_graph* g, bfs_stats* stats, bool timed, int32_t src, bool state_on_host) {
  if (!state_on_host)
    CUDA_TRY(cudaMemcpyAsync(g->h_st, g->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream));
  if (stats && g->persistent)
    CUDA_TRY(cudaMemcpyAsync(g->h_smid, g->d_smid, sizeof(int32_t) * (size_t)g->ctas, cudaMemcpyDeviceToHost,
                             g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  const DevState& st = *g->h_st;
  int rc = traversal_error(st, src);
  if (rc != BFS_OK || !stats) return rc;
  if ((rc = traversal_stats(g, st, g->launches, timed ? g->ev : nullptr, stats)) != BFS_OK) return rc;
  if (stats->per_level && stats->per_level_cap > 0) {
    const int L = std::min(std::min(st.num_levels, stats->per_level_cap), g->lvl_cap);
    if (L > 0)
      CUDA_TRY(cudaMemcpy(stats->per_level, g->d_lvl, sizeof(int32_t) * (size_t)L * kLevelFields,
                          cudaMemcpyDeviceToHost));
    // active SMs: distinct SMs among the CTAs that host the level's warps
    std::vector<int> distinct((size_t)g->ctas + 1, 0);
    if (g->persistent) {
      std::vector<char> seen(4096, 0);
      int cnt = 0;
      for (int b = 0; b < g->ctas; ++b) {
        const int s = g->h_smid[b];
        if (s >= 0 && s < 4096 && !seen[s]) {
          seen[s] = 1;
          ++cnt;
        }
        distinct[b + 1] = cnt;
      }
    }
    for (int l = 0; l < L; ++l) {
      int32_t* r = stats->per_level + (size_t)l * kLevelFields;
      const int ctas = std::min(g->ctas, (r[3] + g->wpc - 1) / g->wpc);
      r[4] = g->persistent ? distinct[ctas] : -1;
      if (!g->persistent) r[5] = r[6] = -1;
    }
  }
  return BFS_OK;
}

static int run_one(bfs_graph* g, int32_t src, int32_t* level_out, int32_t* parent_out, bfs_stats* stats) {
  const bool lvl_dev = is_device_ptr(level_out);
  const bool par_dev = parent_out && is_device_ptr(parent_out);
  // without renumbering the kernels write device outputs in place
  int32_t* level = (lvl_dev && !g->relabel) ? level_out : g->d_level;
  int32_t* parent = (par_dev && !g->relabel) ? parent_out : g->d_parent;
  const Params p = make_params(g, g->relabel ? g->h_inv[src] : src, level, parent);
  const bool timed = stats != nullptr;
  g->launches = 0;
  int rc = enqueue_traversal(g, p, timed ? g->ev : nullptr);
  if (rc != BFS_OK) return rc;
  const int32_t* lvl_src = level;
  const int32_t* par_src = parent;
  if (g->relabel) {
    int32_t* lo = lvl_dev ? level_out : g->d_out_level;
    int32_t* po = parent_out ? (par_dev ? parent_out : g->d_out_parent) : nullptr;
    const int fgrid = std::max(1, std::min(g->sms * 8, (int)(((long long)g->n + kThreads - 1) / kThreads)));
    k_finalize<<<fgrid, kThreads, 0, g->stream>>>(g->n, g->d_inv, g->d_perm, level, parent, lo, po, g->d_st,
                                                  g->h_st_map, p.level_n, p.src);
    CUDA_TRY(cudaGetLastError());
    ++g->launches;
    lvl_src = lo;
    par_src = po;
  }
  if (!lvl_dev)
    CUDA_TRY(cudaMemcpyAsync(level_out, lvl_src, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, g->stream));
  if (parent_out && !par_dev)
    CUDA_TRY(cudaMemcpyAsync(parent_out, par_src, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost,
                             g->stream));
  return finish_traversal(g, stats, timed, src, g->relabel && g->h_st_map);
}

extern "C" int bfs_run(bfs_graph* g, int32_t src, int32_t* level_out, int32_t* parent_out, bfs_stats* stats) {
  if (!g) return fail(BFS_E_INVAL, "graph is NULL");
  if (!level_out) return fail(BFS_E_INVAL, "level_out is NULL");
  if (src < 0 || src >= g->n) return fail(BFS_E_INVAL, "src %d out of range [0, %d)", src, g->n);
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != g->device) CUDA_TRY(cudaSetDevice(g->device));
  const int rc = run_one(g, src, level_out, parent_out, stats);
  if (cur != g->device) cudaSetDevice(cur);
  return rc;
}

extern "C" int bfs_run_frontiers(bfs_graph* g, int32_t src, int32_t* level_out, int32_t* parent_out,
                                 bfs_stats* stats, int32_t* frontiers_out) {
#if !S3BFS_CHECKED
  (void)g;
  (void)src;
  (void)level_out;
  (void)parent_out;
  (void)stats;
  (void)frontiers_out;
  return fail(BFS_E_INVAL, "the frontier dump is part of the checked build (libs3bfs_checked.so)");
#else
  if (!g) return fail(BFS_E_INVAL, "graph is NULL");
  if (!level_out || !frontiers_out) return fail(BFS_E_INVAL, "level_out / frontiers_out is NULL");
  if (src < 0 || src >= g->n) return fail(BFS_E_INVAL, "src %d out of range [0, %d)", src, g->n);
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != g->device) CUDA_TRY(cudaSetDevice(g->device));
  int rc = BFS_OK;
  if (!g->d_fdump) rc = dalloc(g, &g->d_fdump, (size_t)g->n + 4);
  if (rc == BFS_OK) {
    g->fdump_on = true;
    rc = run_one(g, src, level_out, parent_out, stats);
    g->fdump_on = false;
  }
  if (rc == BFS_OK) {
    const size_t r = (size_t)std::min<long long>(g->h_st->reached, g->n);
    CUDA_TRY(cudaMemcpy(frontiers_out, g->d_fdump, sizeof(int32_t) * r, cudaMemcpyDeviceToHost));
    if (g->relabel) {
      std::vector<int32_t> perm((size_t)g->n);
      CUDA_TRY(cudaMemcpy(perm.data(), g->d_perm, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < r; ++i)
        frontiers_out[i] = (unsigned)frontiers_out[i] < (unsigned)g->n ? perm[(size_t)frontiers_out[i]] : -1;
    }
  }
  if (cur != g->device) cudaSetDevice(cur);
  return rc;
#endif
}

// ---- multi-source batches (bitmask frontiers) -----------------------------

static int ms_setup(bfs_graph* g) {
  if (g->ms_ready) return BFS_OK;
  // every buffer is allocated once: a call that failed half-way (memory cap)
  // resumes here without leaking what it got
  int rc;
  const size_t n = (size_t)g->n;
  if (!g->d_seen && (rc = dalloc(g, &g->d_seen, n)) != BFS_OK) return rc;
  if (!g->d_fr[0] && (rc = dalloc(g, &g->d_fr[0], n)) != BFS_OK) return rc;
  if (!g->d_fr[1] && (rc = dalloc(g, &g->d_fr[1], n)) != BFS_OK) return rc;
  // heavy vertices (internal ids), from a host copy of row_ptr
  std::vector<int32_t> rp(n + 1), heavy, huge;
  CUDA_TRY(cudaMemcpy(rp.data(), g->d_row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
  for (size_t v = 0; v < n; ++v) {
    const int32_t d = rp[v + 1] - rp[v];
    if (d > kMsHuge)
      huge.push_back((int32_t)v);
    else if (d > kMsHeavy)
      heavy.push_back((int32_t)v);
  }
  g->n_heavy = (int32_t)heavy.size();
  g->n_huge = (int32_t)huge.size();
  if (!g->d_heavy && (rc = dalloc(g, &g->d_heavy, std::max<size_t>(heavy.size(), 1))) != BFS_OK) return rc;
  if (!g->d_huge && (rc = dalloc(g, &g->d_huge, std::max<size_t>(huge.size(), 1))) != BFS_OK) return rc;
  if (!heavy.empty())
    CUDA_TRY(cudaMemcpy(g->d_heavy, heavy.data(), sizeof(int32_t) * heavy.size(), cudaMemcpyHostToDevice));
  if (!huge.empty())
    CUDA_TRY(cudaMemcpy(g->d_huge, huge.data(), sizeof(int32_t) * huge.size(), cudaMemcpyHostToDevice));
  int per_sm = 0;
  CUDA_TRY(cudaFuncSetAttribute(k_msbfs, cudaFuncAttributeMaxDynamicSharedMemorySize, kMsParentSmem));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_msbfs, kThreads, kMsParentSmem));
  if (per_sm < 1) return fail(BFS_E_CUDA, "multi-source kernel cannot be resident (occupancy 0)");
  g->ms_ctas = per_sm * g->sms;
  if (!g->d_block_or && (rc = dalloc(g, &g->d_block_or, 2 * (size_t)g->ms_ctas)) != BFS_OK) return rc;
  if (!g->d_level_bits && (rc = dalloc(g, &g->d_level_bits, (size_t)g->lvl_cap)) != BFS_OK) return rc;
  if (!g->d_counts && (rc = dalloc(g, &g->d_counts, (size_t)g->ms_ctas * 128)) != BFS_OK) return rc;
  if (!g->d_block_edges && (rc = dalloc(g, &g->d_block_edges, (size_t)g->ms_ctas)) != BFS_OK) return rc;
  if (!g->d_groups && (rc = dalloc(g, &g->d_groups, 3 * 64)) != BFS_OK) return rc;
  if (!g->d_masks && (rc = dalloc(g, &g->d_masks, 64)) != BFS_OK) return rc;
  if (g->ctas < g->ms_ctas) {
    // the barrier's arrival words must cover this grid too
    if (!g->ms_arrive_grown && (rc = dalloc(g, &g->d_arrive, (size_t)(g->ms_ctas + 3) / 4 * 4)) != BFS_OK) return rc;
    g->ms_arrive_grown = true;
  }
  g->ms_ready = true;
  return BFS_OK;
}

// Up to 64 sources in one launch; outputs as for bfs_run_batch.
static int run_group_bitmask(bfs_graph* g, const int32_t* srcs, int k, int32_t* levels_out, int32_t* parents_out,
                             bfs_stats* stats) {
  const size_t n = (size_t)g->n;
  const bool lvl_dev = is_device_ptr(levels_out);
  const bool par_dev = parents_out && is_device_ptr(parents_out);
  int rc;
  if ((!lvl_dev && !g->d_stage_level) && (rc = dalloc(g, &g->d_stage_level, 64 * n)) != BFS_OK) return rc;
  if (parents_out && !par_dev && !g->d_stage_parent && (rc = dalloc(g, &g->d_stage_parent, 64 * n)) != BFS_OK)
    return rc;
  int32_t* L = lvl_dev ? levels_out : g->d_stage_level;
  int32_t* Pp = parents_out ? (par_dev ? parents_out : g->d_stage_parent) : nullptr;
  // sources grouped by (internal) vertex
  int32_t vs[64], src_int[64], src_out[64];
  unsigned long long masks[64];
  int groups = 0;
  for (int i = 0; i < k; ++i) {
    src_out[i] = srcs[i];
    src_int[i] = g->relabel ? g->h_inv[srcs[i]] : srcs[i];
    int j = 0;
    while (j < groups && vs[j] != src_int[i]) ++j;
    if (j == groups) {
      vs[groups] = src_int[i];
      masks[groups++] = 0;
    }
    masks[j] |= 1ull << i;
  }
  int32_t hg[3 * 64];
  memcpy(hg, vs, sizeof(vs));
  memcpy(hg + 64, src_int, sizeof(src_int));
  memcpy(hg + 128, src_out, sizeof(src_out));
  CUDA_TRY(cudaMemcpyAsync(g->d_groups, hg, sizeof(hg), cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaMemcpyAsync(g->d_masks, masks, sizeof(masks), cudaMemcpyHostToDevice, g->stream));
  MsParams p;
  memset(&p, 0, sizeof(p));
  p.n = g->n;
  p.k = k;
  p.row_ptr = g->d_row_ptr;
  p.col_idx = g->d_col_idx;
  p.seen = g->d_seen;
  p.fr[0] = g->d_fr[0];
  p.fr[1] = g->d_fr[1];
  p.heavy = g->d_heavy;
  p.n_heavy = g->n_heavy;
  p.huge = g->d_huge;
  p.n_huge = g->n_huge;
  p.levels_out = L;
  p.parents_out = Pp;
  p.perm = g->relabel ? g->d_perm : nullptr;
  p.inv = g->relabel ? g->d_inv : nullptr;
  p.block_or = g->d_block_or;
  p.level_bits = g->d_level_bits;
  p.block_edges = g->d_block_edges;
  p.lvl_cap = g->lvl_cap;
  p.st = g->d_st;
  p.bar_arrive = g->d_arrive;
  p.spin_ns = g->spin_ns;
  p.debug_flags = 0;
  const bool timed = stats != nullptr;
  if (timed) CUDA_TRY(cudaEventRecord(g->ev[0], g->stream));
  // With few isolated vertices k_msbfs writes every output entry once (-1 for
  // the pairs it never reached); otherwise the outputs are cleared first.  On
  // ER 2^20 the first saves the 83 us clearing pass of a 1.34 ms batch; on
  // R-MAT s22 (43% of the vertices isolated) writing the missing pairs after
  // the pull cost 0.75 ms against 0.54 ms for the clearing pass.
  p.write_missing = (long long)(g->n - g->n_live) * 16 <= (long long)g->n ? 1 : 0;
  if (!p.write_missing) {
    CUDA_TRY(cudaMemsetAsync(L, 0xFF, sizeof(int32_t) * (size_t)k * n, g->stream));
    if (Pp) CUDA_TRY(cudaMemsetAsync(Pp, 0xFF, sizeof(int32_t) * (size_t)k * n, g->stream));
  }
  CUDA_TRY(cudaMemsetAsync(g->d_arrive, 0, sizeof(int32_t) * ((size_t)(g->ms_ctas + 3) / 4 * 4), g->stream));
  const int cgrid = std::max(1, std::min(g->sms * 8, (int)((n + kThreads - 1) / kThreads)));
  k_msbfs_clear<<<cgrid, kThreads, 0, g->stream>>>(p);
  CUDA_TRY(cudaGetLastError());
  k_msbfs_sources<<<1, 64, 0, g->stream>>>(p, g->d_groups, g->d_masks, groups, g->d_groups + 64, g->d_groups + 128);
  CUDA_TRY(cudaGetLastError());
  g->launches = 2;
  if (timed) CUDA_TRY(cudaEventRecord(g->ev[1], g->stream));
  void* args[] = {&p};
  CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_msbfs, dim3(g->ms_ctas), dim3(kThreads), args,
                                       Pp ? kMsParentSmem : 0, g->stream));
  ++g->launches;
  if (timed) CUDA_TRY(cudaEventRecord(g->ev[2], g->stream));
  if (stats) {
    k_msbfs_counts<<<g->ms_ctas, kThreads, 0, g->stream>>>(p, g->d_counts);
    CUDA_TRY(cudaGetLastError());
    ++g->launches;
  }
  if (!lvl_dev)
    CUDA_TRY(cudaMemcpyAsync(levels_out, L, sizeof(int32_t) * (size_t)k * n, cudaMemcpyDeviceToHost, g->stream));
  if (parents_out && !par_dev)
    CUDA_TRY(cudaMemcpyAsync(parents_out, Pp, sizeof(int32_t) * (size_t)k * n, cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaMemcpyAsync(g->h_st, g->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (g->h_st->err == BFS_E_TIMEOUT) return fail(BFS_E_TIMEOUT, "device wait %d ran out (batch)", g->h_st->err_where);
  if (g->h_st->err != 0) return fail(g->h_st->err, "device error %d (batch)", g->h_st->err);
  if (!stats) return BFS_OK;
  float ms_loop = 0.f, ms_all = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms_loop, g->ev[1], g->ev[2]));
  CUDA_TRY(cudaEventElapsedTime(&ms_all, g->ev[0], g->ev[2]));
  const int L_used = std::min(g->h_st->num_levels, g->lvl_cap);
  std::vector<unsigned long long> bits((size_t)std::max(L_used, 1));
  if (L_used > 0)
    CUDA_TRY(cudaMemcpy(bits.data(), g->d_level_bits, sizeof(unsigned long long) * (size_t)L_used,
                        cudaMemcpyDeviceToHost));
  std::vector<long long> counts((size_t)g->ms_ctas * 128), bedges((size_t)g->ms_ctas);
  CUDA_TRY(cudaMemcpy(counts.data(), g->d_counts, sizeof(long long) * counts.size(), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(bedges.data(), g->d_block_edges, sizeof(long long) * bedges.size(), cudaMemcpyDeviceToHost));
  long long work = 0;
  for (long long x : bedges) work += x;
  for (int i = 0; i < k; ++i) {
    bfs_stats& st = stats[i];
    long long reached = 0, edges = 0;
    for (int b = 0; b < g->ms_ctas; ++b) {
      reached += counts[(size_t)b * 128 + i];
      edges += counts[(size_t)b * 128 + 64 + i];
    }
    int levels = 1;
    for (int l = 0; l < L_used; ++l)
      if ((bits[(size_t)l] >> i) & 1ull) levels = l + 2;
    st.num_levels = levels;
    st.active_ctas = g->ms_ctas;
    st.reached = reached;
    st.edges_scanned = edges;
    st.candidates = reached - 1;
    st.ms_level_step = ms_loop;
    st.ms_total = ms_all;
    st.work_edges = work;
    st.launches = g->launches;
  }
  return BFS_OK;
}

// ---- batches of single-source traversals, queued back to back -----------
//
// Traversal i runs on the graph's stream and uses ring slot i % D (D =
// kQueueDepth): its timing events, a pinned copy of its device state block
// and an event that marks it done.  The host queues up to D traversals ahead
// and checks traversal i - D (error, stats) before it reuses that slot, so a
// host that falls behind for a while does not leave the GPU idle.  Device
// outputs are written in place (through k_finalize on a renumbered graph).
// Host outputs go through device staging pair i % S (S = kStagePairs): a
// second stream copies it to the caller's buffers while the next traversals
// run, and traversal i + S waits for that copy on the device before it
// reuses the pair.  With S pairs the traversals can run S - 1 ahead of the
// copies, so a copy that is slow for a while (the device-to-host path is
// shared) delays no traversal as long as the copies keep up on average.
// Copies into pageable host memory are correct but do not overlap.

static int pipe_setup(bfs_graph* g, bool host) {
  int rc;
  if (host)
    for (int s = 0; s < bfs_graph::kStagePairs; ++s) {
      if (!g->d_slot_level[s] && (rc = dalloc(g, &g->d_slot_level[s], (size_t)g->n + 4)) != BFS_OK) return rc;
      if (!g->d_slot_parent[s] && (rc = dalloc(g, &g->d_slot_parent[s], (size_t)g->n + 4)) != BFS_OK) return rc;
    }
  if (g->pipe_ready) return BFS_OK;
  // each handle is created once (a call that failed half-way resumes here)
  for (int s = 0; s < bfs_graph::kQueueDepth; ++s) {
    for (auto& e : g->slot_ev[s])
      if (!e) CUDA_TRY(cudaEventCreate(&e));
    if (!g->slot_ready[s]) CUDA_TRY(cudaEventCreateWithFlags(&g->slot_ready[s], cudaEventDisableTiming));
    if (!g->slot_copied[s]) CUDA_TRY(cudaEventCreateWithFlags(&g->slot_copied[s], cudaEventDisableTiming));
  }
  if (!g->copy_stream) CUDA_TRY(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
  if (!g->h_slot_st &&
      cudaHostAlloc((void**)&g->h_slot_st, bfs_graph::kQueueDepth * sizeof(DevState), cudaHostAllocMapped) !=
          cudaSuccess) {
    cudaGetLastError();
    g->h_slot_st = nullptr;
    return fail(BFS_E_NOMEM, "pinned host allocation failed");
  }
  // k_finalize writes the state blocks through the device's view of them;
  // without one (no mapped pinned memory) they are copied after it instead
  if (!g->h_slot_st_map && cudaHostGetDevicePointer((void**)&g->h_slot_st_map, g->h_slot_st, 0) != cudaSuccess) {
    cudaGetLastError();
    g->h_slot_st_map = nullptr;
  }
  g->pipe_ready = true;
  return BFS_OK;
}

static int run_batch_pipelined(bfs_graph* g, const int32_t* srcs, int32_t k, int32_t* levels_out,
                               int32_t* parents_out, bfs_stats* stats, bool host) {
  constexpr int D = bfs_graph::kQueueDepth;
  int rc = pipe_setup(g, host);
  if (rc != BFS_OK) return rc;
  const size_t n = (size_t)g->n;
  int launches[D] = {};
  // wait for traversal i (and its copy), then check it
  auto finish = [&](int32_t i) -> int {
    const int s = i % D;
    CUDA_TRY(cudaEventSynchronize(host ? g->slot_copied[s] : g->slot_ready[s]));
    const DevState& st = g->h_slot_st[s];
    int r = traversal_error(st, srcs[i]);
    if (r == BFS_OK && stats) r = traversal_stats(g, st, launches[s], g->slot_ev[s], stats + i);
    return r;
  };
  int32_t failed = -1, done = 0;  // traversals [0, done) are checked
  for (int32_t i = 0; i < k && rc == BFS_OK; ++i) {
    if (i >= D) {
      // ring slot i % D is free once traversal i - D is checked
      if ((rc = finish(done)) != BFS_OK) {
        failed = done;
        break;
      }
      ++done;
    }
    constexpr int S = bfs_graph::kStagePairs;
    const int s = i % D, b = i % S;
    if (host && i >= S) CUDA_TRY(cudaStreamWaitEvent(g->stream, g->slot_copied[(i - S) % D], 0));
    // this traversal's outputs on the device, and its working arrays
    int32_t* lo = host ? g->d_slot_level[b] : levels_out + (size_t)i * n;
    int32_t* po = parents_out ? (host ? g->d_slot_parent[b] : parents_out + (size_t)i * n) : nullptr;
    int32_t* lw = g->relabel ? g->d_level : lo;
    int32_t* pw = (g->relabel || !po) ? g->d_parent : po;
    const Params p = make_params(g, g->relabel ? g->h_inv[srcs[i]] : srcs[i], lw, pw);
    g->launches = 0;
    rc = enqueue_traversal(g, p, stats ? g->slot_ev[s] : nullptr);
    if (rc != BFS_OK) {
      failed = i;
      break;
    }
    if (g->relabel) {
      const int fgrid = std::max(1, std::min(g->sms * 8, (int)(((long long)g->n + kThreads - 1) / kThreads)));
      k_finalize<<<fgrid, kThreads, 0, g->stream>>>(g->n, g->d_inv, g->d_perm, lw, pw, lo, po, g->d_st,
                                                    g->h_slot_st_map ? g->h_slot_st_map + s : nullptr, p.level_n,
                                                    p.src);
      CUDA_TRY(cudaGetLastError());
      ++g->launches;
    }
    launches[s] = g->launches;
    if (!g->relabel || !g->h_slot_st_map)
      CUDA_TRY(cudaMemcpyAsync(&g->h_slot_st[s], g->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaEventRecord(g->slot_ready[s], g->stream));
    if (host) {
      CUDA_TRY(cudaStreamWaitEvent(g->copy_stream, g->slot_ready[s], 0));
      CUDA_TRY(cudaMemcpyAsync(levels_out + (size_t)i * n, lo, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                               g->copy_stream));
      if (po)
        CUDA_TRY(cudaMemcpyAsync(parents_out + (size_t)i * n, po, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                 g->copy_stream));
      CUDA_TRY(cudaEventRecord(g->slot_copied[s], g->copy_stream));
    }
  }
  while (rc == BFS_OK && done < k) {
    if ((rc = finish(done)) != BFS_OK) failed = done;
    ++done;
  }
  if (rc != BFS_OK) {
    // nothing of this call stays in flight
    cudaStreamSynchronize(g->stream);
    cudaStreamSynchronize(g->copy_stream);
    if (failed >= 0) {
      char keep[sizeof(g_last_error) - 32];
      snprintf(keep, sizeof(keep), "%.*s", (int)sizeof(keep) - 1, g_last_error);
      snprintf(g_last_error, sizeof(g_last_error), "source index %d: %s", failed, keep);
    }
  }
  return rc;
}

extern "C" int bfs_run_batch(bfs_graph* g, const int32_t* srcs, int32_t k, int32_t* levels_out,
                             int32_t* parents_out, bfs_stats* stats) {
  if (!g) return fail(BFS_E_INVAL, "graph is NULL");
  if (k < 0 || (k > 0 && (!srcs || !levels_out))) return fail(BFS_E_INVAL, "bad batch arguments (k = %d)", k);
  for (int32_t i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->n) return fail(BFS_E_INVAL, "srcs[%d] = %d out of range", i, srcs[i]);
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != g->device) CUDA_TRY(cudaSetDevice(g->device));
  int rc = BFS_OK;
  if (g->symmetric && g->batch_bitmask >= 0 && k >= 2) {
    // groups of up to 64 sources share one bitmask traversal
    rc = ms_setup(g);
    for (int32_t i = 0; i < k && rc == BFS_OK; i += 64) {
      const int kk = std::min(64, k - i);
      rc = run_group_bitmask(g, srcs + i, kk, levels_out + (size_t)i * g->n,
                             parents_out ? parents_out + (size_t)i * g->n : nullptr, stats ? stats + i : nullptr);
    }
    if (cur != g->device) cudaSetDevice(cur);
    return rc;
  }
  // traversals queued back to back (host outputs: copies overlapped), unless
  // per-level records are wanted or the outputs mix device and host memory
  bool per_level = false;
  for (int32_t i = 0; stats && i < k; ++i) per_level |= stats[i].per_level && stats[i].per_level_cap > 0;
  const bool lvl_dev = is_device_ptr(levels_out);
  if (k >= 2 && g->persistent && !per_level && (!parents_out || is_device_ptr(parents_out) == lvl_dev)) {
    rc = run_batch_pipelined(g, srcs, k, levels_out, parents_out, stats, !lvl_dev);
    if (cur != g->device) cudaSetDevice(cur);
    return rc;
  }
  for (int32_t i = 0; i < k && rc == BFS_OK; ++i) {
    rc = run_one(g, srcs[i], levels_out + (size_t)i * g->n, parents_out ? parents_out + (size_t)i * g->n : nullptr,
                 stats ? stats + i : nullptr);
    if (rc != BFS_OK) {
      char keep[sizeof(g_last_error) - 32];
      snprintf(keep, sizeof(keep), "%.*s", (int)sizeof(keep) - 1, g_last_error);
      snprintf(g_last_error, sizeof(g_last_error), "source index %d: %s", i, keep);
    }
  }
  if (cur != g->device) cudaSetDevice(cur);
  return rc;
}

// ---------------------------------------------------------------------------
// bfs_run_csr_noalloc: one traversal that allocates nothing
// ---------------------------------------------------------------------------
//
// For callers that cannot allocate device memory while they traverse: code
// embedded in a host framework whose caching allocator owns the GPU's memory
// (a second allocator would fragment its pool or push it over its budget),
// and latency-critical loops where cudaMalloc / cudaFree would synchronise the
// device and stall other streams.  The caller passes the CSR and the outputs;
// all working memory sits in one file-scope device array of fixed maximum
// size, which every GPU that loads this library's device code reserves until
// the process exits.  Maximum: kNoAllocMaxN vertices, kNoAllocMaxNnz edges.

constexpr int kNoAllocMaxN = 1 << 18;     // 262,144 vertices
constexpr int kNoAllocMaxNnz = 1 << 21;   // 2,097,152 directed edges
constexpr int kNoAllocMaxCtas = 2048;     // cap of the persistent grid
constexpr int kNoAllocMaxDevices = 64;

constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNaState = 0;
constexpr size_t kNaBad = na_align(sizeof(DevState));
constexpr size_t kNaArrive = kNaBad + 256;
constexpr size_t kNaSmid = kNaArrive + na_align(sizeof(int32_t) * kNoAllocMaxCtas);
constexpr size_t kNaStatus = kNaSmid + na_align(sizeof(int32_t) * kNoAllocMaxCtas);
constexpr size_t kNaFront = kNaStatus + na_align(sizeof(ChunkStatus) * kNoAllocMaxCtas * 32);
constexpr size_t kNaFrontOne = na_align(sizeof(int32_t) * (kNoAllocMaxN + 4));
constexpr size_t kNaCol = kNaFront + 6 * kNaFrontOne;
constexpr size_t kNaCand = kNaCol + na_align(sizeof(int32_t) * (kNoAllocMaxNnz + 8));
constexpr size_t kNaAux = kNaCand + na_align(sizeof(int2) * (kNoAllocMaxNnz + 32));
constexpr size_t kNoAllocScratchBytes = kNaAux + na_align(sizeof(int32_t) * (kNoAllocMaxNnz + 32));

// The scratch itself (about 40 MB).  Host code must not use this name as an
// address: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  bool ready;
  unsigned char* scratch;  // device address of g_noalloc_scratch on this device
  int ctas;
  int sms;
};
static NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;
// held for a whole call: calls from different host threads on one device
// would otherwise overlap on the GPU and race on the shared array
static std::mutex g_noalloc_call_mu[kNoAllocMaxDevices];

// Per-device set-up, done by the first call on each device with that device
// current: look up the scratch address and the persistent grid size.
static int noalloc_setup(int dev, NoAllocDevice** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr)
      return fail(BFS_E_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    int sms = 0, coop = 0, per_sm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return fail(BFS_E_CUDA, "device %d has no cooperative launch", dev);
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level_loop<32, false>, 32 * kWarp, loop_smem(0)));
    if (per_sm < 1) return fail(BFS_E_CUDA, "level-loop kernel cannot be resident (occupancy 0)");
    d.scratch = static_cast<unsigned char*>(ptr);
    d.sms = sms;
    d.ctas = std::min(per_sm * sms, kNoAllocMaxCtas);
    d.ready = true;
  }
  *out = &d;
  return BFS_OK;
}

extern "C" int bfs_run_csr_noalloc(int32_t n, int32_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                                   int32_t src, int32_t* level_out, int32_t* parent_out, void* cuda_stream) {
  if (n < 1 || n > kNoAllocMaxN)
    return fail(BFS_E_INVAL, "n = %d: the allocation-free entry point takes 1..%d vertices", n, kNoAllocMaxN);
  if (nnz < 0 || nnz > kNoAllocMaxNnz)
    return fail(BFS_E_INVAL, "nnz = %d: the allocation-free entry point takes 0..%d edges", nnz, kNoAllocMaxNnz);
  if (!row_ptr || (nnz > 0 && !col_idx) || !level_out || !parent_out)
    return fail(BFS_E_INVAL, "NULL pointer argument");
  if (src < 0 || src >= n) return fail(BFS_E_INVAL, "src %d out of range [0, %d)", src, n);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(BFS_E_INVAL, "device %d beyond %d", dev, kNoAllocMaxDevices);
  std::lock_guard<std::mutex> call_lock(g_noalloc_call_mu[dev]);
  NoAllocDevice* d = nullptr;
  int rc = noalloc_setup(dev, &d);
  if (rc != BFS_OK) return rc;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* s = d->scratch;
  int32_t* col = reinterpret_cast<int32_t*>(s + kNaCol);
  int* bad = reinterpret_cast<int*>(s + kNaBad);

  // copy col_idx into the aligned, padded scratch copy that the 16-byte quad
  // loads read; then the range checks every later access relies on
  CUDA_TRY(cudaMemsetAsync(col + (nnz & ~3), 0, sizeof(int32_t) * 8, stream));
  if (nnz > 0)
    CUDA_TRY(cudaMemcpyAsync(col, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, stream));
  CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), stream));
  const int cgrid = std::max(1, std::min(d->sms * 8, (int)(((long long)std::max(n, nnz) + 255) / 256)));
  k_check_csr<<<cgrid, 256, 0, stream>>>(n, nnz, row_ptr, col, bad);
  CUDA_TRY(cudaGetLastError());
  int h_bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (h_bad == 1) return fail(BFS_E_INVAL, "row_ptr must start at 0, never decrease and end at nnz");
  if (h_bad == 2) return fail(BFS_E_INVAL, "col_idx entry out of range [0, n)");

  Params p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  p.nnz = nnz;
  p.row_ptr = row_ptr;
  p.col_idx = col;
  p.level = level_out;
  p.parent = parent_out;
  for (int b = 0; b < 2; ++b) {
    p.F[b] = reinterpret_cast<int32_t*>(s + kNaFront + (size_t)(3 * b + 0) * kNaFrontOne);
    p.RS[b] = reinterpret_cast<int32_t*>(s + kNaFront + (size_t)(3 * b + 1) * kNaFrontOne);
    p.EX[b] = reinterpret_cast<int32_t*>(s + kNaFront + (size_t)(3 * b + 2) * kNaFrontOne);
  }
  p.cand = reinterpret_cast<int2*>(s + kNaCand);
  p.cand_aux = reinterpret_cast<int32_t*>(s + kNaAux);
  p.cand_cnt = nullptr;
  p.status = reinterpret_cast<ChunkStatus*>(s + kNaStatus);
  p.bar_arrive = reinterpret_cast<int32_t*>(s + kNaArrive);
  p.cta_smid = reinterpret_cast<int32_t*>(s + kNaSmid);
  p.st = reinterpret_cast<DevState*>(s + kNaState);
  p.lvl = nullptr;
  p.lvl_cap = 0;
  p.grain = 64;
  p.work_insensitive = 0;
  p.src = src;
  p.max_chunks = d->ctas * 32;
  p.debug_flags = 0;
  p.spin_ns = 1000000000ll;
  p.hub_bits = nullptr;
  p.hub_n = 0;
  p.small_edges = 256 * 32;

  // k_init clears the look-back and barrier state left by the previous call
  const int igrid = std::max(1, std::min(d->sms, (int)(((long long)n / 4 + kThreads - 1) / kThreads)));
  k_init<<<igrid, kThreads, 0, stream>>>(p, d->ctas);
  CUDA_TRY(cudaGetLastError());
  void* args[] = {&p};
  CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_level_loop<32, false>, dim3(d->ctas), dim3(32 * kWarp), args, loop_smem(0),
                                       stream));
  DevState h;
  CUDA_TRY(cudaMemcpyAsync(&h, p.st, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (h.err == BFS_E_TIMEOUT) return fail(BFS_E_TIMEOUT, "device wait %d ran out (src %d)", h.err_where, src);
  if (h.err == BFS_E_MULTIGRAPH)
    return fail(BFS_E_MULTIGRAPH, "next frontier larger than n: the graph repeats a neighbour (src %d)", src);
  if (h.err != 0) return fail(h.err, "device error %d at %d (src %d)", h.err, h.err_where, src);
  return BFS_OK;
}
