// Serving: many single-source traversals, possibly on different graphs, in
// one cooperative launch, advanced level by level.
//
// Every running query owns a slot: the Params of its traversal (its graph's
// CSR, its own level/parent/frontier/candidate buffers and control block).
// At every level all CTAs compute the same split of the grid among the
// running queries -- each gets at least one CTA and the rest in proportion to
// its level's edge count -- and each CTA runs the S3BFS level step (explore,
// grid barrier, compact with a scan over that query's CTAs, grid barrier) for
// its query.  A launch returns after a bounded number of levels or as soon as
// a query finishes, so that the host can retire finished queries and admit
// new ones between launches (continuous batching at level granularity).
// Batching queries is not in the paper; each query is Parallel-BFS(s, P)
// (Fig. 1) unchanged.
#pragma once

#include "s3bfs_device.cuh"

namespace s3bfs {

constexpr int kMaxSlots = 128;

struct SlotDev {
  Params p;            // the query's traversal
  int32_t level;       // its current level
  int32_t active;      // 1 while it runs, 0 when done (or failed)
  int32_t num_levels;  // levels done
  int32_t pad;
  int32_t n, e;        // frontier size and edge count of the current level (copies of the
                       // query's control block, read by every CTA at every step in one load)
  long long reached, edges, cands;
};

struct ServeParams {
  SlotDev* slots;
  int32_t nslots;
  int32_t max_levels;  // levels per launch
  int32_t grain;
  // a query with one CTA and a level of at most local_edges edges runs up to
  // local_levels levels per step alone, with CTA barriers (0: off)
  int32_t local_levels;
  int32_t local_edges;
  int32_t* finished;   // set when a query finished during this launch
  // host-mapped flag: set by a submission while the launch runs, so that the
  // launch returns after its current step and the query gets admitted
  const volatile int32_t* wake;
  // grid barrier state of the server
  DevState* st;
  int32_t* bar_arrive;
  long long spin_ns;
  int32_t debug_flags;
};

// Split of gridDim.x CTAs among the running queries: every query with a
// non-empty frontier gets one CTA plus a share of the rest proportional to
// its level's edge count.  Whole CTA (the slot states are read in parallel,
// one thread per slot, and kept in shared memory: s_lne[q] = level, n, e of
// query q); thread 0 then sets q (-1: idle CTA, -2: nothing runs -- also
// when the step before asked the launch to end), the CTA's rank in its
// query's group and the group size.
__device__ __forceinline__ void serve_assign(const ServeParams& sp, long long* s_w, int3* s_lne, int* q_out,
                                             int* rank_out, int* size_out, bool check_finished) {
  const int t = threadIdx.x;
  __shared__ int s_stop;
  if (t < sp.nslots) {
    const SlotDev& sd = sp.slots[t];
    const int act = ld_relaxed(&sd.active);
    const int lv = ld_relaxed(&sd.level);
    const int n = ld_relaxed(&sd.n);
    const int e = ld_relaxed(&sd.e);
    s_w[t] = act && n > 0 ? (long long)max(e, 1) : 0ll;
    s_lne[t] = make_int3(lv, n, e);
  }
  if (t == kMaxSlots - 1) s_stop = check_finished ? ld_relaxed(sp.finished) : 0;
  __syncthreads();
  if (t == 0) {
    const int G = gridDim.x;
    long long wsum = 0;
    int A = 0;
    for (int q = 0; q < sp.nslots; ++q) {
      wsum += s_w[q];
      A += s_w[q] > 0;
    }
    *q_out = (A == 0 || s_stop != 0) ? -2 : -1;
    const long long spare = G > A ? G - A : 0;
    int start = 0;
    for (int q = 0; q < sp.nslots && A > 0 && s_stop == 0; ++q) {
      if (s_w[q] == 0) continue;
      const int g = 1 + (int)(spare * s_w[q] / wsum);
      if ((int)blockIdx.x >= start && (int)blockIdx.x < start + g) {
        *q_out = q;
        *rank_out = (int)blockIdx.x - start;
        *size_out = g;
      }
      start += g;
    }
  }
}

// Levels of one query run by this CTA alone (the query got one CTA and its
// levels are small): explore, CTA barrier, compaction, CTA barrier, slot
// update, up to sp.local_levels levels or until a level is no longer small or
// the query ends.  The rest of the grid meanwhile runs its own queries' level
// and waits at the step's grid barrier.
template <int W>
__device__ void serve_local(const ServeParams& sp, SlotDev* sd) {
  __shared__ int s_go;
  const Params& p = sd->p;
  const int wib = threadIdx.x >> 5;
  for (int k = 0; k < sp.local_levels; ++k) {
    const int l = ld_relaxed(&sd->level);
    const int par = l & 1;
    const int n_l = ld_relaxed(&sd->n);
    const int e_l = ld_relaxed(&sd->e);
    if (n_l <= 0 || e_l > sp.local_edges) break;  // uniform: every thread read the same words
    int P_l, C_l;
    level_sizing(e_l, W, sp.grain, 0, &P_l, &C_l);
    int cnt = 0, e_begin = 0, work = 0;
    if (wib < P_l) {
      const long long eb = (long long)wib * C_l;
      e_begin = (int)min(eb, (long long)e_l);
      const int e_end = (int)min(eb + C_l, (long long)e_l);
      work = e_end - e_begin;
      if (e_begin < e_end) cnt = explore_chunk<W>(p, l, par, n_l, e_l, e_begin, e_end, p.cand + e_begin, nullptr, 0);
    }
    __syncthreads();
    if (P_l == 0) {
      if (threadIdx.x == 0) publish_empty_next(p, par);
    } else {
      compact_cta<W>(p, l, par, P_l, p.cand + e_begin, p.cand_aux + e_begin, cnt, 0, work);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int n_next = ld_relaxed(&p.st->ctrl[par ^ 1].n);
      sd->reached += n_l;
      sd->edges += e_l;
      sd->cands += ld_relaxed(&p.st->ctrl[par ^ 1].c);
      sd->num_levels = l + 1;
      st_relaxed(&sd->n, n_next);
      st_relaxed(&sd->e, ld_relaxed(&p.st->ctrl[par ^ 1].e));
      st_relaxed(&sd->level, l + 1);
      const bool done = n_next <= 0 || ld_relaxed(&p.st->err) != 0;
      if (done) {
        st_relaxed(&sd->active, 0);
        st_relaxed(sp.finished, 1);
      }
      s_go = !done;
    }
    __syncthreads();
    if (!s_go) break;
  }
}

// One launch: up to sp.max_levels levels of every running query.
template <int W>
__global__ void __launch_bounds__(W * kWarp, W == 8 ? 4 : 1) k_serve(ServeParams sp) {
  __shared__ int s_q, s_rank, s_size;
  __shared__ long long s_w[kMaxSlots];
  __shared__ int3 s_lne[kMaxSlots];
  const int wib = threadIdx.x >> 5;
  const bool watch = blockIdx.x == 0 && threadIdx.x == 0 && sp.wake != nullptr;
  init_cta_err();
  int bar = 0;
  for (int it = 0; it < sp.max_levels; ++it) {
    // read early: the host-memory load overlaps the step's work
    const int woke = watch ? *sp.wake : 0;
    // the finished flag of the step before is read with the slot states
    serve_assign(sp, s_w, s_lne, &s_q, &s_rank, &s_size, it > 0);
    __syncthreads();
    const int q = s_q, rank = s_rank, gsize = s_size;
    __syncthreads();
    if (q == -2) break;  // same decision in every CTA: they read the same slot states
    SlotDev* sd = q >= 0 ? sp.slots + q : nullptr;
    // a query alone on this CTA with a small level: several levels now, alone
    bool local = false;
    if (sd && gsize == 1 && sp.local_levels > 0) local = ld_relaxed(&sd->e) <= sp.local_edges;
    if (local) {
      serve_local<W>(sp, sd);
      sd = nullptr;  // nothing left for this step's shared phases
    }
    int l = 0, par = 0, n_l = 0, e_l = 0, P_l = 0, C_l = 0, cnt = 0, e_begin = 0, work = 0;
    if (sd) {
      const Params& p = sd->p;
      l = s_lne[q].x;
      par = l & 1;
      n_l = s_lne[q].y;
      e_l = s_lne[q].z;
      level_sizing(e_l, gsize * W, sp.grain, 0, &P_l, &C_l);
      const int gw = rank * W + wib;
      if (gw < P_l) {
        const long long eb = (long long)gw * C_l;
        e_begin = (int)min(eb, (long long)e_l);
        const int e_end = (int)min(eb + C_l, (long long)e_l);
        work = e_end - e_begin;
        if (e_begin < e_end)
          cnt = explore_chunk<W>(p, l, par, n_l, e_l, e_begin, e_end, p.cand + e_begin, nullptr, 0);
      }
    }
    if (!grid_sync(sp, ++bar, kSleepBusy, false)) break;
    if (sd) {
      const Params& p = sd->p;
      if (P_l == 0) {
        if (rank == 0 && threadIdx.x == 0) publish_empty_next(p, par);
      } else if (rank * W < P_l) {
        compact_cta<W>(p, l, par, P_l, p.cand + e_begin, p.cand_aux + e_begin, cnt, rank, work);
      }
      // the CTA that published the next level's sizes updates the slot
      const int last = P_l == 0 ? 0 : (P_l - 1) / W;
      if (rank == last && threadIdx.x == 0) {
        const int n_next = ld_relaxed(&p.st->ctrl[par ^ 1].n);
        sd->reached += n_l;
        sd->edges += e_l;
        sd->cands += ld_relaxed(&p.st->ctrl[par ^ 1].c);
        sd->num_levels = l + 1;
        st_relaxed(&sd->n, n_next);
        st_relaxed(&sd->e, ld_relaxed(&p.st->ctrl[par ^ 1].e));
        st_relaxed(&sd->level, l + 1);
        if (n_next <= 0 || ld_relaxed(&p.st->err) != 0) {
          st_relaxed(&sd->active, 0);
          st_relaxed(sp.finished, 1);
        }
      }
    }
    if (woke) st_relaxed(sp.finished, 1);  // a query waits: end after this step
    if (!grid_sync(sp, ++bar, kSleepBusy, false)) break;
    // a finished query or a waiting one ends the launch at the next step's
    // assignment (retire and admit before going on)
  }
}

}  // namespace s3bfs
