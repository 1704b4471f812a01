// Host-side internals shared by the library's translation units: the graph
// object behind the opaque bfs_graph handle, error reporting and device
// allocation helpers.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "s3bfs.h"
#include "s3bfs_device.cuh"

using s3bfs::ChunkStatus;
using s3bfs::DevState;

struct bfs_graph {
  int device = 0;
  cudaStream_t stream = nullptr;
  int32_t n = 0, nnz = 0;
  int sms = 0;
  int ctas = 0;   // G
  int warps = 0;  // P
  int wpc = 32;   // warps per CTA of the level loop (8 or 32)
  int grain = 64;
  int persistent = 1;
  int work_insensitive = 0;
  int debug_flags = 0;
  long long spin_ns = 1000000000ll;
  int small_edges = -1;  // resolved at create: 256 edges per warp of one CTA
  int launches = 0;      // kernels launched by the current call
  int direction = 0;     // 1: direction-optimising (bottom-up levels)
  int alpha = 15, beta = 18, gamma = 2;
  int32_t n_live = 0;    // vertices of degree > 0
  int32_t nwords = 0;    // words of a frontier bitmap
  uint32_t* d_fb[2] = {nullptr, nullptr};
  int32_t *d_ulist = nullptr, *d_ulist_cnt = nullptr;  // bottom-up: unvisited vertices per warp
  int32_t lvl_cap = 0;
  int hub_n = 0;         // vertices [0, hub_n) have visited bits in shared memory
  bool relabel = false;  // internal ids are degree-descending (hubs first)
  std::vector<int32_t> h_inv;
  int32_t *d_perm = nullptr, *d_inv = nullptr;
  uint32_t* d_hub_bits = nullptr;
  int32_t *d_out_level = nullptr, *d_out_parent = nullptr;  // translated outputs for host buffers
  int32_t *d_row_ptr = nullptr, *d_col_idx = nullptr;
  int32_t *d_level = nullptr, *d_parent = nullptr;
  int32_t *d_F[2] = {nullptr, nullptr}, *d_RS[2] = {nullptr, nullptr}, *d_EX[2] = {nullptr, nullptr};
  int2* d_cand = nullptr;
  int32_t* d_cand_aux = nullptr;
  int32_t* d_cand_cnt = nullptr;
  ChunkStatus* d_status = nullptr;
  int32_t *d_arrive = nullptr, *d_smid = nullptr;
  DevState* d_st = nullptr;
  int32_t* d_lvl = nullptr;
  DevState* h_st = nullptr;      // pinned
  DevState* h_st_map = nullptr;  // the device's pointer to h_st, if mapped
  int32_t* h_smid = nullptr; // pinned
  int32_t* h_ctrl = nullptr; // pinned, launch-per-phase mode
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  std::vector<void*> allocs;
  size_t dev_bytes = 0;  // device memory allocated through dalloc
  size_t dev_cap = 0;    // bfs_opts.max_device_bytes (0 = no cap)
  bool ms_arrive_grown = false;  // bitmask batches widened the barrier's arrival words
  int32_t* d_fdump = nullptr;    // checked build: frontiers of one traversal in level order
  bool fdump_on = false;
  // multi-source (bitmask) batches, allocated at the first batch
  bool symmetric = false;
  int batch_bitmask = 0;
  bool ms_ready = false;
  int ms_ctas = 0;
  unsigned long long *d_seen = nullptr, *d_fr[2] = {nullptr, nullptr};
  int32_t *d_heavy = nullptr, *d_huge = nullptr;
  int32_t n_heavy = 0, n_huge = 0;
  unsigned long long *d_block_or = nullptr, *d_level_bits = nullptr;
  long long* d_block_edges = nullptr;
  long long* d_counts = nullptr;
  int32_t* d_groups = nullptr;  // vs[64], src_int[64], src_out[64]
  unsigned long long* d_masks = nullptr;
  int32_t *d_stage_level = nullptr, *d_stage_parent = nullptr;  // 64 x n, for host outputs
  // batches of single-source traversals queued back to back: a ring of
  // kQueueDepth slots (events, pinned state block) lets the host run that many
  // traversals ahead; with host outputs also one device staging pair (level,
  // parent) per slot, whose copy to the host overlaps the traversals after it
  static constexpr int kQueueDepth = 8;
  static constexpr int kStagePairs = kQueueDepth;
  bool pipe_ready = false;
  cudaStream_t copy_stream = nullptr;
  int32_t *d_slot_level[kStagePairs] = {}, *d_slot_parent[kStagePairs] = {};
  cudaEvent_t slot_ev[kQueueDepth][3] = {};
  cudaEvent_t slot_ready[kQueueDepth] = {}, slot_copied[kQueueDepth] = {};
  DevState* h_slot_st = nullptr;      // pinned [kQueueDepth]
  DevState* h_slot_st_map = nullptr;  // the device's pointer to h_slot_st, if mapped
};

// last error text of this host thread (bfs_last_error) and its setter
extern thread_local char g_last_error[512];
int fail(int code, const char* fmt, ...);

#define CUDA_TRY(expr)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) return fail(BFS_E_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                     \
  } while (0)

template <class T>
inline int dalloc(bfs_graph* g, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (g->dev_cap && g->dev_bytes + bytes > g->dev_cap)
    return fail(BFS_E_NOMEM, "device memory cap: %zu bytes allocated, %zu more would pass max_device_bytes = %zu",
                g->dev_bytes, bytes, g->dev_cap);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(BFS_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  g->allocs.push_back(q);
  g->dev_bytes += bytes;
  *p = static_cast<T*>(q);
  return BFS_OK;
}

// true for device (or managed) memory; host pointers, pinned or not, are false
bool is_device_ptr(const void* p);

