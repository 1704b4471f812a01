// Kernels of the S3BFS level loop (GB300, sm_103a): init, the persistent
// level loop (top-down levels; bottom-up levels in the direction-optimising
// variant), the launch-per-phase explore / compact kernels, the CSR check and
// the translation of a renumbered graph's outputs.  Device building blocks:
// s3bfs_device.cuh.  Included once, by s3bfs.cu.
#pragma once

#include "s3bfs_device.cuh"

using namespace s3bfs;

// a0 (Fig. 1, initialisation): level = parent = -1 except level[s] = 0, parent[s] =
// s; F_0 = [s] with its row start and degree; clear the scan and barrier state.
__global__ void __launch_bounds__(kThreads) k_init(Params p, int ctas) { init_traversal(p, ctas); }

// The whole level loop runs in one cooperative launch (k_level_loop).  A
// level with at most p.small_edges edges starts a streak that CTA 0 runs
// alone while the levels stay that small (the others wait at one grid
// barrier); every other level runs on the whole grid.  Warps beyond P_l skip
// the level's work and wait at the barrier, so a small level occupies few SMs.
//
// One level of the loop (explore, barrier, compact, barrier).  GRID: all
// CTAs with grid barriers.  Otherwise CTA 0 alone, its warps taking the
// chunks, with CTA barriers (small levels).  Returns false if the traversal
// must stop (an error, including a wait that ran out).
//
// s_ctrl (shared memory) holds the control block of level l for CTA 0 while
// it runs small levels alone: it reads the level's sizes from there and the
// compaction leaves the next level's there, so a small level makes no round
// trip to global memory for them; the global error word is then read every
// 32 levels (an error this CTA raises itself shows in s_ctrl).
template <int W>
__device__ __forceinline__ bool one_level(const Params& p, int l, int n_l, int e_l, int* bar, uint32_t* s_hub,
                                       long long* acc, bool GRID, LevelCtrl* s_ctrl) {
  __shared__ int s_err;
  const int lane = threadIdx.x & (kWarp - 1);
  const int gw = GRID ? blockIdx.x * W + (threadIdx.x >> 5) : (threadIdx.x >> 5);
  const int P = GRID ? gridDim.x * W : W;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const int par = l & 1;
  int P_l, C_l;
  level_sizing(e_l, P, p.grain, p.work_insensitive, &P_l, &C_l);
  long long t_level = 0;
  if (leader) {
    t_level = global_ns();
    acc[0] += n_l;
    acc[1] += e_l;
    record_level(p, l, n_l, e_l, P_l);
  }
  // big level: take the visited-bits snapshot into shared memory
  const int hub_lim = (GRID && p.hub_n > 0 && e_l >= p.hub_n) ? load_hub_bits(p, s_hub) : 0;
  int cnt = 0, e_begin = 0, work = 0;
  if (gw < P_l) {
    const long long eb = (long long)gw * C_l;
    e_begin = (int)min(eb, (long long)e_l);
    const int e_end = (int)min(eb + C_l, (long long)e_l);
    work = e_end - e_begin;
    if (e_begin < e_end) cnt = explore_chunk<W>(p, l, par, n_l, e_l, e_begin, e_end, p.cand + e_begin, s_hub, hub_lim);
  }
  // a CTA without a chunk in this level waits with a longer back-off
  const bool idle = (int)blockIdx.x * W >= P_l;
  if (GRID) {
    if (!grid_sync(p, ++*bar, idle ? kSleepIdle : kSleepBusy)) return false;
  } else {
    __syncthreads();
  }
  if (leader && l < p.lvl_cap) p.lvl[(long long)l * kLevelFields + 6] = (int)min(global_ns() - t_level, 2147483647ll);
  if (GRID && p.hub_n > 0) build_hub_bits(p, gw, P);
  if (P_l == 0) {
    if (gw == 0 && lane == 0) {
      publish_empty_next(p, par);
      if (!GRID) *s_ctrl = LevelCtrl{0, 0, 0, s_ctrl->cum, 0, 0, 0, s_ctrl->vcum};
    }
  } else if (!GRID || (int)blockIdx.x * W < P_l) {
    compact_cta<W>(p, l, par, P_l, p.cand + e_begin, p.cand_aux + e_begin, cnt, GRID ? (int)blockIdx.x : 0, work,
                   GRID ? nullptr : s_ctrl);
  }
  if (GRID) {
    // (the next level may give every CTA work: no back-off here)
    if (!grid_sync(p, ++*bar)) return false;
  } else {
    __syncthreads();
    if ((l & 31) == 31) {
      if (threadIdx.x == 0) s_err = ld_relaxed(&p.st->err);
      __syncthreads();
      if (s_err != 0) return false;
    }
    if (s_ctrl->n < 0) return false;
  }
  if (leader) {
    acc[2] += GRID ? ld_relaxed(&p.st->ctrl[par ^ 1].c) : s_ctrl->c;
    acc[3] += GRID ? ld_relaxed(&p.st->ctrl[par ^ 1].w) : s_ctrl->w;
    if (l < p.lvl_cap) p.lvl[(long long)l * kLevelFields + 5] = (int)min(global_ns() - t_level, 2147483647ll);
  }
  return true;
}

// One bottom-up level on the whole grid (direction-optimising traversal of a
// symmetric graph).  After a top-down level the frontier bitmap is first
// built from the level array (grid barrier) and every vertex word is
// scanned; after a bottom-up level only the warps' unvisited lists are.
// Then (grid barrier) the next level's frontier bitmap is built from the
// level array while the standard compaction turns the new vertices into the
// next frontier record and publishes its sizes (grid barrier).  Warp gw's
// candidates and unvisited list use its own region: room for the 128
// vertices of every group of four bitmap words it owns.
template <int W>
__device__ __noinline__ bool bu_level(const Params& p, int l, int n_l, int e_l, int* bar, long long* acc) {
  const int gw = blockIdx.x * W + (threadIdx.x >> 5);
  const int P = gridDim.x * W;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const int par = l & 1;
  uint32_t* fb_cur = par ? p.fb[1] : p.fb[0];
  uint32_t* fb_next = par ? p.fb[0] : p.fb[1];
  long long t_level = 0;
  if (leader) {
    t_level = global_ns();
    acc[0] += n_l;
    acc[1] += e_l;
    record_level(p, l, n_l, e_l, P, 1);
  }
  const bool after_bu = ld_relaxed(&p.st->ctrl[par].fb) != 0;
#if S3BFS_BU_BITMAP
  if (!after_bu) {
    build_frontier_bits(p, l, fb_cur, gw, P);
    if (!grid_sync(p, ++*bar)) return false;
  }
#endif
  // warp gw's region: 128 entries per 128-vertex group it owns
  const int gpw = (p.bu_groups + P - 1) / P;
  const long long base = (long long)gw * gpw * 128;
  int work = 0, first = 0, work0 = 0;
  const int total = after_bu ? ld_relaxed(p.ulist_cnt + gw)
                             : bu_unvisited(p, l, fb_cur, gw, P, p.ulist + base, p.cand + base, &first, &work0);
  const int cnt = first + bu_scan(p, l, fb_cur, gw, total, p.ulist + base, p.cand + base + first, &work,
                                  after_bu ? 0 : 1);
  work += __reduce_add_sync(0xffffffffu, work0);
  if (!grid_sync(p, ++*bar)) return false;
  if (leader && l < p.lvl_cap) p.lvl[(long long)l * kLevelFields + 6] = (int)min(global_ns() - t_level, 2147483647ll);
#if S3BFS_BU_BITMAP
  build_frontier_bits(p, l + 1, fb_next, gw, P);
#else
  (void)fb_next;
#endif
  if (p.hub_n > 0) build_hub_bits(p, gw, P);
  compact_cta<W>(p, l, par, P, p.cand + base, p.cand_aux + base, cnt, (int)blockIdx.x, work);
  if (!grid_sync(p, ++*bar)) return false;
  if (leader) {
    acc[2] += ld_relaxed(&p.st->ctrl[par ^ 1].c);
    acc[3] += ld_relaxed(&p.st->ctrl[par ^ 1].w);
    if (l < p.lvl_cap) p.lvl[(long long)l * kLevelFields + 5] = (int)min(global_ns() - t_level, 2147483647ll);
  }
  return true;
}

// 8-warp CTAs: four per SM (64 registers a thread); wider CTAs: one per SM
// (64, 80 or 128 registers a thread with 32, 24 or 16 warps)
template <int W, bool DO>
__global__ void __launch_bounds__(W * kWarp, W == 8 ? 4 : 1) k_level_loop(Params p) {
  extern __shared__ __align__(16) uint32_t s_hub[];  // visited bits, p.hub_n / 8 bytes
  const int gw = blockIdx.x * W + (threadIdx.x >> 5);
  const int P = gridDim.x * W;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  if (threadIdx.x == 0) p.cta_smid[blockIdx.x] = sm_id();
  init_cta_err();
  __shared__ LevelCtrl s_ctrl;  // CTA 0 during a streak: the current level's control block
  int bar = 0, l = 0;
  long long acc[4] = {0, 0, 0, 0};  // reached, edges, candidates, work (leader)
  bool streak = false;           // CTA 0 is running small levels alone
  while (true) {
    int n_l, e_l;
    bool bottom_up;
    if (streak) {
      n_l = s_ctrl.n;
      e_l = s_ctrl.e;
      bottom_up = s_ctrl.dir != 0;
    } else {
      n_l = ld_relaxed(&p.st->ctrl[l & 1].n);
      e_l = ld_relaxed(&p.st->ctrl[l & 1].e);
      bottom_up = ld_relaxed(&p.st->ctrl[l & 1].dir) != 0;
    }
    const bool small = n_l > 0 && p.small_edges > 0 && e_l <= p.small_edges && !bottom_up;
    if (streak && !small) {
      // CTA 0 ends its streak: the whole grid resumes at level l (or stops)
      streak = false;
      if (threadIdx.x == 0) st_relaxed(&p.st->resume_level, l);
      if (!grid_sync(p, ++bar)) break;
      if (p.hub_n > 0) {
        // the visited bits were not kept up to date by the streak
        build_hub_bits(p, gw, P);
        if (!grid_sync(p, ++bar)) break;
      }
      continue;
    }
    if (n_l <= 0) break;
    if (l + 2 >= (int)kEpochMask) {
      if (leader) set_err(p, BFS_E_INVAL, 5);
      break;
    }
    if (small && blockIdx.x != 0) {
      // parked at one grid barrier while CTA 0 runs the small levels
      if (!grid_sync(p, ++bar, kSleepParked)) break;
      l = ld_relaxed(&p.st->resume_level);
      if (p.hub_n > 0) {
        build_hub_bits(p, gw, P);
        if (!grid_sync(p, ++bar)) break;
      }
      continue;
    }
    if (DO && bottom_up) {
      if (!bu_level<W>(p, l, n_l, e_l, &bar, acc)) break;
      ++l;
      continue;
    }
    if (small && !streak) {
      // a streak starts: its control blocks live in shared memory
      if (threadIdx.x == 0) {
        const LevelCtrl* c = &p.st->ctrl[l & 1];
        s_ctrl = LevelCtrl{n_l, e_l, 0, ld_relaxed(&c->cum), 0, 0, 0, ld_relaxed(&c->vcum)};
      }
      __syncthreads();
    }
    streak = small;
    if (!one_level<W>(p, l, n_l, e_l, &bar, s_hub, acc, !small, &s_ctrl)) {
      if (streak) {
        // release the parked CTAs; the error word makes everybody stop
        if (threadIdx.x == 0) st_relaxed(&p.st->resume_level, l);
        grid_sync(p, ++bar);
      }
      break;
    }
    ++l;
    if (small && threadIdx.x == 0) st_relaxed(&p.st->progress, l);
  }
  if (leader) {
    p.st->num_levels = l;
    p.st->reached = acc[0];
    p.st->edges = acc[1];
    p.st->cands = acc[2];
    p.st->work = acc[3];
  }
}

// Launch-per-phase mode: the same two phases as separate launches; the host
// reads n and e of the next level in between.
template <int W>
__global__ void __launch_bounds__(W * kWarp) k_explore(Params p, int l, int n_l, int e_l, int P_l, int C_l) {
  const int gw = blockIdx.x * W + (threadIdx.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) record_level(p, l, n_l, e_l, P_l);
  if (gw >= P_l) return;
  const long long eb = (long long)gw * C_l;
  const int e_begin = (int)min(eb, (long long)e_l);
  const int e_end = (int)min(eb + C_l, (long long)e_l);
  int cnt = 0;
  if (e_begin < e_end) cnt = explore_chunk<W>(p, l, l & 1, n_l, e_l, e_begin, e_end, p.cand + e_begin, nullptr, 0);
  if ((threadIdx.x & (kWarp - 1)) == 0) p.cand_cnt[gw] = cnt;
}

template <int W>
__global__ void __launch_bounds__(W * kWarp) k_compact(Params p, int l, int e_l, int P_l, int C_l) {
  const int gw = blockIdx.x * W + (threadIdx.x >> 5);
  const int par = l & 1;
  if (P_l == 0) {
    if (gw == 0 && (threadIdx.x & (kWarp - 1)) == 0) publish_empty_next(p, par);
    return;
  }
  // every thread of the CTA takes part; warps without a chunk bring 0
  const int e_begin = gw < P_l ? (int)min((long long)gw * C_l, (long long)e_l) : 0;
  const int e_end = gw < P_l ? (int)min((long long)gw * C_l + C_l, (long long)e_l) : 0;
  const int cnt = gw < P_l ? ld_relaxed(&p.cand_cnt[gw]) : 0;
  compact_cta<W>(p, l, par, P_l, p.cand + e_begin, p.cand_aux + e_begin, cnt, (int)blockIdx.x, e_end - e_begin);
}

// CSR sanity checks that every traversal relies on (no out-of-range access):
// row_ptr starts at 0, never decreases, ends at nnz; 0 <= col_idx < n.
__global__ void k_check_csr(int32_t n, int32_t nnz, const int32_t* rp, const int32_t* ci, int* bad) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (tid == 0 && (rp[0] != 0 || rp[n] != nnz)) *bad = 1;
  for (long long i = tid; i < n; i += stride)
    if (rp[i] > rp[i + 1]) *bad = 1;
  for (long long e = tid; e < nnz; e += stride)
    if ((unsigned)ci[e] >= (unsigned)n) *bad = 2;
}

// Outputs of a renumbered graph back in the caller's vertex ids: v is the
// caller's id, inv[v] the internal one, perm[i] the caller's id of internal i.
// With st_host set (a device-mapped pointer to pinned host memory), block 0
// also copies the finished traversal's state block there, so no copy-engine
// transfer has to sit between this kernel and the next traversal's.
__global__ void __launch_bounds__(kThreads) k_finalize(int32_t n, const int32_t* inv, const int32_t* perm,
                                                       const int32_t* level, const int32_t* parent,
                                                       int32_t* level_out, int32_t* parent_out,
                                                       const DevState* st, DevState* st_host, int32_t n_kept,
                                                       int32_t s) {
  static_assert(sizeof(DevState) % sizeof(int32_t) == 0, "state block is copied in words");
  if (st_host && blockIdx.x == 0)
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(int32_t)); w += blockDim.x)
      reinterpret_cast<int32_t*>(st_host)[w] = reinterpret_cast<const int32_t*>(st)[w];
  finalize_outputs(n, inv, perm, level, parent, level_out, parent_out, n_kept, s);
}
