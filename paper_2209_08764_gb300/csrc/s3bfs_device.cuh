// S3BFS level step on sm_103a: device code.
//
// One level of Parallel-BFS (one pass of Fig. 1's main loop) runs as two phases separated
// by a grid-wide barrier:
//
//   EXPLORE  (Fig. 1, thread count to EXPLORE-VERTEX)  the level's e_l edges are split into P_l chunks of
//            C_l = ceil(e_l / P_l) consecutive edges, one chunk per warp, with
//            P_l = min(P, ceil(e_l / grain)) (Fig. 1's thread count; grain = 1 is the paper's
//            formula).  A warp finds its start (frontier entry, edge offset) by
//            a search on the exclusive degree scan EX (Find-StartExpPoint), then walks its
//            edges: for an edge (u, v) with level[v] == -1 it stores
//            level[v] = l + 1 and parent[v] = u with plain (relaxed, non-RMW)
//            stores and emits the candidate pair (v, u) into its own region of
//            the candidate buffer (EXPLORE-VERTEX; Algorithm section).
//   COMPACT  (Fig. 1, owner check to linearisation)  each warp re-reads parent[v] for its candidates and
//            keeps (v, u) iff parent[v] == u: the owner of v is the vertex
//            whose store to parent[v] landed last, so exactly one candidate
//            per newly reached v survives (Fig. 1's owner check, with the owner id taken
//            to be the parent vertex).  A single-pass decoupled look-back scan
//            over the chunks, in chunk order, gives every survivor its slot in
//            the next frontier (Sizes prefix sum, linearisation) and, in the same pass, the
//            exclusive prefix sum of the survivors' degrees, i.e. the next
//            level's degree gather and EdgeSum scan.
//
// The next frontier is stored as three int32 arrays: F (vertex), RS (first CSR
// position of its row) and EX (exclusive degree prefix, with EX[n] = e).
// No atomic read-modify-write instruction is used anywhere: the paper's BFS
// takes neither locks nor atomic instructions (Abstract).  Cross-warp
// ordering uses release/acquire stores and loads only.
#pragma once

#include <cstdint>

#include "s3bfs.h"

// Build-time knobs (tuning experiments).
#ifndef S3BFS_LEVEL_CACHED
#define S3BFS_LEVEL_CACHED 1  // 1: level[v] tests through L1 (weak loads), 0: relaxed loads at L2
#endif
#ifndef S3BFS_COL_EVICT_FIRST
#define S3BFS_COL_EVICT_FIRST 1  // 1: col_idx streamed with an L2 evict-first policy, no L1 allocation
#endif
#ifndef S3BFS_QPL
#define S3BFS_QPL 2  // col_idx quads per lane per round of the explore walk
#endif
#ifndef S3BFS_CR
#define S3BFS_CR 2  // candidates per lane per batch of the compaction
#endif
#ifndef S3BFS_WPC
#define S3BFS_WPC 32  // warps per CTA of the auxiliary kernels (init, finalize, bitmask batches)
#endif
#ifndef S3BFS_HUB_LOG2
#define S3BFS_HUB_LOG2 18  // visited bits in shared memory for up to 2^this vertices
#endif

namespace s3bfs {

constexpr int kWarp = 32;
constexpr int kWarpsPerCta = S3BFS_WPC;
constexpr int kThreads = kWarp * kWarpsPerCta;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kLevelFields = BFS_LEVEL_FIELDS;
// visited bits in shared memory cover at most this many vertices
constexpr int kHubMax = 1 << S3BFS_HUB_LOG2;
// hard iteration cap of every spin-wait, on top of the time limit
constexpr int kSpinIters = 1 << 21;

constexpr unsigned long long kFlagAgg = 1ull;
constexpr unsigned long long kFlagIncl = 2ull;
constexpr unsigned kEpochMask = 0x3FFFFFFFu;

// Scan state of one CTA of a level: word = [63:62] flag, [61:32] epoch
// (level+1), [31:0] kept count; the degree and candidate sums sit in slots
// written before the word is released.
struct alignas(32) ChunkStatus {
  unsigned long long word;
  int32_t agg_deg, agg_cand, agg_work;
  int32_t pad[3];
};

// Sizes of the frontier of one level, published by the compaction of the
// level before (by parity of the level).
struct LevelCtrl {
  int32_t n, e;  // frontier size n_l and its edge count e_l
  int32_t c;     // candidates the level before emitted
  int32_t cum;   // e summed over this level and all earlier ones (<= nnz)
  int32_t dir;   // how this level runs: 0 top-down, 1 bottom-up
  int32_t fb;    // 1: the level before wrote this level's frontier bitmap
  int32_t w;     // neighbour entries the level before examined
  int32_t vcum;  // n summed over this level and all earlier ones (vertices visited)
};

// Device-resident control block of one traversal.
struct DevState {
  LevelCtrl ctrl[2];  // size n and edge count e of the frontier of level l, by parity of l
  int32_t err;        // 0 or a BFS_E_* code
  int32_t err_where;  // which wait or check failed
  int32_t num_levels;
  int32_t bar_release;
  long long reached, edges, cands;
  int32_t progress;      // levels done by CTA 0 alone (the others wait; progress extends their wait)
  int32_t resume_level;  // level at which the whole grid resumes after CTA 0 ran small levels alone
  long long work;        // neighbour entries examined, all levels
};

struct Params {
  int32_t n, nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;  // padded: readable up to a multiple of 4 entries past nnz
  int32_t* level;
  int32_t* parent;
  // 1: parent[] is not cleared at init (parent[s] = s only).  Allowed when
  // nothing reads the parent of an unreached vertex: the dedup reads only
  // vertices claimed in the level, and the outputs pass through
  // finalize_outputs, which reads a parent only where the level is >= 0.
  int32_t parent_lazy;
  int32_t* F[2];
  int32_t* RS[2];
  int32_t* EX[2];
  int2* cand;           // candidate pairs (v, u); chunk k owns [k*C_l, (k+1)*C_l)
  int32_t* cand_aux;    // per candidate slot: degree prefix of a stashed survivor
  int32_t* cand_cnt;    // per chunk, for the launch-per-phase mode
  ChunkStatus* status;  // per CTA
  int32_t* bar_arrive;  // per CTA
  int32_t* cta_smid;    // per CTA
  DevState* st;
  int32_t* lvl;         // per-level statistics, lvl_cap x kLevelFields
  int32_t lvl_cap;
  int32_t grain;
  int32_t work_insensitive;
  int32_t src;
  int32_t max_chunks;   // size of status / cand_cnt
  int32_t debug_flags;
  long long spin_ns;
  // visited bits of vertices [0, hub_n) (hub_n a multiple of 128, 0 = none):
  // rebuilt from level[] after every level's explore, copied to shared memory
  // at the start of a level with at least hub_n edges
  uint32_t* hub_bits;
  int32_t hub_n;
  // levels with at most this many edges run on CTA 0 alone, with CTA barriers
  // instead of grid barriers (0 = never)
  int32_t small_edges;
  // direction-optimising traversal of a symmetric graph: bottom-up levels
  // test neighbours against the frontier bitmap fb[l & 1] (bit v set iff
  // level[v] == l) and write the next level's bitmap fb[(l + 1) & 1]
  uint32_t* fb[2];
  int32_t nwords;     // words of a frontier bitmap: ceil(n / 32), padded to a multiple of 4
  // 128-vertex groups a bottom-up level scans for unvisited vertices: all
  // (nwords / 4), or on a graph renumbered by descending degree only those up
  // to the last vertex of degree > 0 (the isolated ones come last and no
  // level ever reaches them)
  int32_t bu_groups;
  // level entries a traversal clears and finalize_outputs reads: n, or on a
  // graph renumbered by descending degree (parent_lazy) the vertices of
  // degree > 0, which come first (no edge reaches the isolated ones; 0 = n)
  int32_t level_n;
  // per warp: the vertices still unvisited after a bottom-up level (in the
  // warp's region, like its candidates) and their count
  int32_t* ulist;
  int32_t* ulist_cnt;
  int32_t direction;  // 0: every level top-down; 1: direction-optimising
  int32_t alpha, beta, gamma;
  int32_t n_live;     // vertices of degree > 0 (the ones a bottom-up level can find)
  // 1: the start-point search first probes the entries around
  // e_begin * n_l / e_l (graphs of near-uniform degree, where EX is close to
  // linear in the entry index); 0: plain 32-ary search (skewed graphs)
  int32_t guess_search;
#if S3BFS_CHECKED
  // checked build: every frontier in level order (F_0, F_1, ...), n entries
  // (null: no dump)
  int32_t* fdump;
#endif
};

// ---------------------------------------------------------------------------
// memory operations (inline PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// relaxed load without a compiler memory barrier (hot loop: the loads only
// need to be single-copy atomic, not ordered against other accesses)
__device__ __forceinline__ int ld_relaxed_nb(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// L2-coherent loads of data written before the last grid barrier
__device__ __forceinline__ int ld_cg(const int* p) {
  int v;
  asm volatile("ld.global.cg.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int2 ld_cg2(const int2* p) {
  int2 v;
  asm volatile("ld.global.cg.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
// 128-bit read-only load of four consecutive col_idx entries
__device__ __forceinline__ int4 ld_nc4(const int4* p) {
  int4 v;
  asm volatile("ld.global.nc.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_cg4u(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ int4 ld_relaxed4(const int4* p) {
  int4 v;
  asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
// level[v] test of the explore walk.  Within a level a stale -1 only adds a
// duplicate candidate (removed by the dedup); across levels the acquire at
// the grid barrier makes every earlier write visible.
__device__ __forceinline__ int ld_level(const int* p) {
#if S3BFS_LEVEL_CACHED
  int v;
  asm volatile("ld.global.ca.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
#else
  return ld_relaxed_nb(p);
#endif
}
__device__ __forceinline__ unsigned long long col_policy() {
  unsigned long long pol = 0;
#if S3BFS_COL_EVICT_FIRST
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#endif
  return pol;
}
__device__ __forceinline__ int4 ld_col4(const int4* p, unsigned long long pol) {
#if S3BFS_COL_EVICT_FIRST
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
#else
  (void)pol;
  return ld_nc4(p);
#endif
}
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int sm_id() {
  int s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

// Per-CTA flag in shared memory: this CTA raised an error.  Its next grid
// barrier arrival carries it, so the barrier learns of the error without a
// read of the global error word.  Every kernel that uses grid_sync clears it
// at its start (init_cta_err).
__device__ __forceinline__ int& cta_err_flag() {
  __shared__ int f;
  return f;
}
__device__ __forceinline__ void init_cta_err() {
  if (threadIdx.x == 0) cta_err_flag() = 0;
  __syncthreads();
}

// Raise an error (the first one raised stays: a later error is a consequence).
template <class P>
__device__ __forceinline__ void set_err(const P& p, int code, int where) {
  cta_err_flag() = 1;
  if (ld_relaxed(&p.st->err) != 0) return;
  st_relaxed(&p.st->err_where, where);
  st_relaxed(&p.st->err, code);
}

// Checked build (S3BFS_CHECKED=1, a debug library of its own): an index
// outside its array sets BFS_E_CHECK with the check's id in err_where and
// the access is skipped, so nothing faults; every CTA then leaves at its
// next barrier.  The production build compiles every check away.
#ifndef S3BFS_CHECKED
#define S3BFS_CHECKED 0
#endif
template <class P>
__device__ __forceinline__ bool in_range(const P& p, long long i, long long cap, int where) {
#if S3BFS_CHECKED
  if (i >= 0 && i < cap) return true;
  set_err(p, BFS_E_CHECK, where);
  return false;
#else
  (void)p;
  (void)i;
  (void)cap;
  (void)where;
  return true;
#endif
}

__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const int t = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += t;
  }
  return x;
}

// P_l and C_l of a level (Fig. 1's thread count, with a grain; Algorithm section:
// a near-equal split of the e_l edges).  Shared by host and device.
__host__ __device__ inline void level_sizing(int e_l, int P, int grain, int work_insensitive, int* P_l,
                                             int* C_l) {
  if (e_l <= 0) {
    *P_l = 0;
    *C_l = 0;
    return;
  }
  long long p = work_insensitive ? P : ((long long)e_l + grain - 1) / grain;
  if (p > P) p = P;
  if (p < 1) p = 1;
  *P_l = (int)p;
  *C_l = (int)(((long long)e_l + p - 1) / p);
}

// ---------------------------------------------------------------------------
// grid barrier without atomics: every CTA publishes its arrival in its own
// word; CTA 0 waits for all of them, then releases one word everybody waits
// on.  The release word carries the error state: 2 * epoch + 1 when any CTA
// raised an error before the barrier (or CTA 0's wait failed), so the
// waiting CTAs learn it without another load.  Every wait is bounded by the
// time limit and an iteration cap; on expiry the error word is set and all
// CTAs return false.  Returns false, in every CTA, when any CTA raised an
// error before the barrier.
// ---------------------------------------------------------------------------
// sleep_cap: the longest pause between two polls of the release word by a
// waiting CTA (ns).  A CTA with work polls every 64 ns; a CTA with nothing
// to do before the release backs off exponentially up to the cap: up to
// 512 ns for a CTA without a chunk in a level (the phase after the release
// takes several microseconds, so a late wake-up delays nobody), 2048 ns for
// one parked while CTA 0 runs a streak of small levels.
constexpr int kSleepBusy = 64;
constexpr int kSleepIdle = 512;
constexpr int kSleepParked = 2048;
// flagged: the CTAs' error flags ride on their arrival words (every error
// raised in the launch concerns p.st).  A launch whose CTAs also raise errors
// that must not stop the grid (per-query errors of the query server) passes
// false: CTA 0 then reads p.st->err once the arrivals are in.
template <class P>
__device__ bool grid_sync(const P& p, int epoch, int sleep_cap = kSleepBusy, bool flagged = true) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool stall =
        (p.debug_flags & BFS_DEBUG_STALL_BARRIER) && epoch == 1 && blockIdx.x == gridDim.x - 1;
    __threadfence();
    // arrival word: 2 * epoch, + 1 if this CTA raised an error
    if (!stall) st_relaxed(&p.bar_arrive[blockIdx.x], 2 * epoch + (flagged && cta_err_flag() ? 1 : 0));
  }
  const unsigned target = (unsigned)epoch;
  if (blockIdx.x == 0) {
    // CTA 0 gathers the arrivals, four words per 16-byte load (the arrival
    // array is padded to a multiple of four entries); an arrival's low bit
    // says that CTA raised an error before it arrived
    bool ok = true, raised = false;
    const long long t0 = global_ns();
    const int groups = ((int)gridDim.x + 3) >> 2;
    const int4* arr4 = reinterpret_cast<const int4*>(p.bar_arrive);
    const int e2 = 2 * epoch;
    for (int q = threadIdx.x; q < groups && ok; q += blockDim.x) {
      const int base = q << 2;
      int it = 0;
      while (true) {
        const int4 a = ld_relaxed4(arr4 + q);
        const bool done = (a.x >= e2 || base + 0 >= (int)gridDim.x) && (a.y >= e2 || base + 1 >= (int)gridDim.x) &&
                          (a.z >= e2 || base + 2 >= (int)gridDim.x) && (a.w >= e2 || base + 3 >= (int)gridDim.x);
        if (done) {
          raised |= ((a.x & 1) && base + 0 < (int)gridDim.x) || ((a.y & 1) && base + 1 < (int)gridDim.x) ||
                    ((a.z & 1) && base + 2 < (int)gridDim.x) || ((a.w & 1) && base + 3 < (int)gridDim.x);
          break;
        }
        ++it;
        if ((it & 31) == 0 && ld_relaxed(&p.st->err) != 0) {
          ok = false;
          break;
        }
        if (it > kSpinIters || global_ns() - t0 > p.spin_ns) {
          set_err(p, BFS_E_TIMEOUT, 1);
          ok = false;
          break;
        }
        if (it > 64) __nanosleep(64);
      }
    }
    ok = __syncthreads_and(ok && !raised);
    if (threadIdx.x == 0) {
      __threadfence();  // the arrivals seen above happen before the error check; the release after this CTA's writes
      const bool err = !ok || (flagged ? cta_err_flag() != 0 : ld_relaxed(&p.st->err) != 0);
      st_relaxed(&p.st->bar_release, (int)(2u * target + (err ? 1u : 0u)));
      s_ok = !err;
    }
  } else if (threadIdx.x == 0) {
    int ok = 1, it = 0, nap = kSleepBusy;
    long long t0 = global_ns();
    int prog = ld_relaxed(&p.st->progress);
    while (true) {
      const unsigned r = (unsigned)ld_acquire(&p.st->bar_release);
      if ((r >> 1) >= target) {
        ok = (r & 1u) == 0;
        break;
      }
      ++it;
      if ((it & 31) == 0) {
        if (ld_relaxed(&p.st->err) != 0) {
          ok = 0;
          break;
        }
        // CTA 0 working alone through small levels is progress, not a stall
        const int pr = ld_relaxed(&p.st->progress);
        if (pr != prog) {
          prog = pr;
          t0 = global_ns();
          it = 0;
        }
      }
      if (it > kSpinIters || global_ns() - t0 > p.spin_ns) {
        set_err(p, BFS_E_TIMEOUT, 2);
        ok = 0;
        break;
      }
      if (it > 64) {
        __nanosleep(nap);
        nap = min(2 * nap, sleep_cap);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// EXPLORE: one warp, edges [e_begin, e_end) of level l
// ---------------------------------------------------------------------------

// Append the candidates flagged in this lane slot, in lane order.
__device__ __forceinline__ int emit(int2* out, int cnt, bool k, int v, int u, int lane) {
  const unsigned m = __ballot_sync(kFull, k);
  if (k) out[cnt + __popc(m & ((1u << lane) - 1u))] = make_int2(v, u);
  return cnt + __popc(m);
}

// Returns the number of candidate pairs written to out (warp-uniform).
// s_hub / hub_lim: visited bits of vertices [0, hub_lim) in shared memory, a
// snapshot taken at the start of the level (hub_lim = 0: none).  A set bit
// means the vertex already has a level, so its level[] test is skipped.
#ifndef S3BFS_EXPLORE_QUAL
#define S3BFS_EXPLORE_QUAL inline
#endif
#ifndef S3BFS_PPL
#define S3BFS_PPL 1  // probes per lane in a round of the start-point search (1: 32-ary)
#endif
#ifndef S3BFS_OWNER_REDUX
#define S3BFS_OWNER_REDUX 1  // 1: quad owners by ballot + OR-reduction and shared records; 0: shuffle search
#endif
template <int W>  // warps per CTA
__device__ S3BFS_EXPLORE_QUAL int explore_chunk(const Params& p, int l, int par, int n_l, int e_l, int e_begin,
                                                int e_end,
                             int2* out, const uint32_t* s_hub, int hub_lim) {
  const int lane = threadIdx.x & (kWarp - 1);
#if S3BFS_OWNER_REDUX
  __shared__ int4 s_rec[W][kWarp];
  int4* rec = s_rec[threadIdx.x >> 5];
  const unsigned lane_lt = (1u << lane) - 1u;
#endif
  // (selects, not p.EX[par]: a runtime index into the parameter block would
  // copy it to local memory)
  const int* EX = par ? p.EX[1] : p.EX[0];
  const int* F = par ? p.F[1] : p.F[0];
  const int* RS = par ? p.RS[1] : p.RS[0];
  const int4* col4 = reinterpret_cast<const int4*>(p.col_idx);
  int* level = p.level;
  int* parent = p.parent;
  const int lnext = l + 1;
  const unsigned long long pol = col_policy();

  // Find-StartExpPoint (Fig. 1): the last frontier entry i with EX[i] <=
  // e_begin (upper bound minus one), by a 32-ary search -- every round the
  // lanes probe 32 evenly spaced entries of [lo, hi) and keep the last probe
  // that is still <= e_begin.  Invariant: EX[lo] <= e_begin < EX[hi].
  int lo = 0, hi = n_l;
  if (p.guess_search && n_l > kWarp) {
    // one round around the proportional guess first: 32 consecutive entries
    // (every 32nd entry on a level of more than kGuessWide entries).  The
    // probes only shrink [lo, hi) and keep the invariant; on a near-uniform
    // degree they bracket the start, which leaves one step (or none).
    constexpr int kGuessWide = 8192;
    const int s = n_l > kGuessWide ? kWarp : 1;
    const long long g0 = (long long)e_begin * n_l / e_l - (long long)(kWarp / 2) * s;
    const long long x = min(max(g0 + (long long)lane * s, 0ll), (long long)n_l - 1);
    // positions never decrease with the lane, so the probes <= e_begin are a prefix
    const int c = __popc(__ballot_sync(kFull, in_range(p, x, n_l + 1, 10) && ld_cg(EX + x) <= e_begin));
    const int x_first = __shfl_sync(kFull, (int)x, 0);
    const int x_le = __shfl_sync(kFull, (int)x, max(c - 1, 0));
    const int x_gt = __shfl_sync(kFull, (int)x, min(c, kWarp - 1));
    if (c == 0) {
      hi = x_first;  // > 0: EX[0] = 0 <= e_begin
    } else if (c == kWarp) {
      lo = x_le;
    } else {
      lo = x_le;
      hi = x_gt;
    }
  }
  while (hi - lo > 1) {
    // S3BFS_PPL probes per lane a round (lane L probes PPL*L .. PPL*L + PPL - 1)
    constexpr int kPpl = S3BFS_PPL;
    constexpr int kProbes = kPpl * kWarp;
    const int step = (hi - lo + kProbes - 1) / kProbes;
    int cntle = 0;
#pragma unroll
    for (int t = 0; t < kPpl; ++t) {
      const int idx = lo + (kPpl * lane + t) * step;
      cntle += (idx < hi && in_range(p, idx, n_l + 1, 10) && ld_cg(EX + idx) <= e_begin) ? 1 : 0;
    }
    // probes are in increasing order and EX is non-decreasing, so the probes
    // <= e_begin form a prefix: its length minus one is the last such probe
    const int J = __reduce_add_sync(kFull, cntle) - 1;
    lo += J * step;
    hi = min(lo + step, hi);
  }

  int i = lo;  // current frontier entry
  int e = e_begin;
  int cnt = 0;
  // A window of 32 frontier entries, one per lane: its first edge EX[idx],
  // the edge after its last EX[idx+1], its row start and vertex.  The next
  // window's loads are issued as soon as its start is known (right after the
  // current window is staged), so they run under the current window's walk.
  bool pf_in;
  int pf_lo, pf_hi, pf_rs, pf_u;
  {
    const int idx = i + lane;
    pf_in = idx < n_l && in_range(p, n_l, (long long)p.n + 1, 11) && in_range(p, idx, p.n, 12);
    pf_lo = pf_in ? ld_cg(EX + idx) : e_l;
    pf_hi = (pf_in && lane == kWarp - 1) ? ld_cg(EX + idx + 1) : e_l;
    pf_rs = pf_in ? ld_cg(RS + idx) : 0;
    pf_u = pf_in ? ld_cg(F + idx) : 0;
  }
  while (e < e_end) {
    const bool in = pf_in;
    const int ex_lo = pf_lo;
    int ex_hi = __shfl_down_sync(kFull, ex_lo, 1);
    if (lane == kWarp - 1) ex_hi = pf_hi;
    const int rs = pf_rs;
    const int u = pf_u;
    const int tile_end = min(e_end, __shfl_sync(kFull, ex_hi, kWarp - 1));
    // the next window starts past the entries whose edges this one finishes
    const int i_next = i + __popc(__ballot_sync(kFull, in && ex_hi <= tile_end));
    if (tile_end < e_end) {
      const int idx = i_next + lane;
      pf_in = idx < n_l && in_range(p, idx, p.n, 12);
      pf_lo = pf_in ? ld_cg(EX + idx) : e_l;
      pf_hi = (pf_in && lane == kWarp - 1) ? ld_cg(EX + idx + 1) : e_l;
      pf_rs = pf_in ? ld_cg(RS + idx) : 0;
      pf_u = pf_in ? ld_cg(F + idx) : 0;
    }
    // This lane's edges inside the tile, as CSR positions [p0, p1), covered by
    // the 16-byte aligned quads q0 .. q0+nq-1 of col_idx.
    const int a = max(ex_lo, e), b = min(ex_hi, tile_end);
    int p0 = 0, p1 = 0, q0 = 0, nq = 0;
    if (in && a < b) {
      p0 = rs + (a - ex_lo);
      p1 = rs + (b - ex_lo);
      q0 = p0 >> 2;
      nq = ((p1 - 1) >> 2) - q0 + 1;
    }
    const int qend = warp_incl_scan(nq, lane);
    const int Q = __shfl_sync(kFull, qend, kWarp - 1);
    const int qoff = qend - nq;
#if S3BFS_OWNER_REDUX
    // The entries that own quads, packed by rank into the warp's shared
    // records: quad q of the window lies at col_idx quad R.x + q and belongs
    // to edges [R.y, R.z) of vertex R.w.
    __syncwarp();
    const unsigned nzm = __ballot_sync(kFull, nq > 0);
    if (nq > 0) rec[__popc(nzm & lane_lt)] = make_int4(q0 - qoff, p0, p1, u);
    __syncwarp();
#endif
    // Load-balanced walk: round r hands quad r*32+lane to this lane; its owner
    // entry w is the first lane whose quad range ends after it.
    for (int base = 0; base < Q; base += kWarp * S3BFS_QPL) {
      int4 c[S3BFS_QPL];
      int wp0[S3BFS_QPL], wp1[S3BFS_QPL], wu[S3BFS_QPL], pos[S3BFS_QPL];
#pragma unroll
      for (int r = 0; r < S3BFS_QPL; ++r) {
        const int q = base + r * kWarp + lane;
        bool act = q < Q;
#if S3BFS_OWNER_REDUX
        // owner rank of quad q: the entries ending at or before the block
        // start B, plus those ending inside (B, q] (one bit each: quad ranges
        // of non-empty entries end at distinct positions)
        const int B = base + r * kWarp;
        const int wB = __popc(__ballot_sync(kFull, nq > 0 && qend <= B));
        const unsigned endbit = (nq > 0 && qend > B && qend < B + kWarp) ? 1u << (qend - B - 1) : 0u;
        const unsigned ends = __reduce_or_sync(kFull, endbit);
        const int w = min(wB + __popc(ends & lane_lt), kWarp - 1);
        const int4 R = rec[w];  // (a lane past Q may read a record this launch never wrote)
        const int qa = R.x + q;
        act = act && in_range(p, qa, ((long long)p.nnz + 7) >> 2, 13);
        wp0[r] = R.y;
        wp1[r] = act ? R.z : 0;  // no valid position on a lane past Q
        wu[r] = R.w;
#else
        int w = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
          const int t = __shfl_sync(kFull, qend, w + s - 1);
          if (t <= q) w += s;
        }
        const int wq0 = __shfl_sync(kFull, q0, w);
        const int wqoff = __shfl_sync(kFull, qoff, w);
        wp0[r] = __shfl_sync(kFull, p0, w);
        wp1[r] = __shfl_sync(kFull, p1, w);
        wu[r] = __shfl_sync(kFull, u, w);
        const int qa = wq0 + (q - wqoff);
        act = act && in_range(p, qa, ((long long)p.nnz + 7) >> 2, 13);
#endif
        c[r] = make_int4(0, 0, 0, 0);
        if (act) c[r] = ld_col4(col4 + qa, pol);
        pos[r] = act ? (qa << 2) : 0x7FFFFFF0;   // inactive: no position is valid
      }
      int lv[S3BFS_QPL][4];
      bool vv[S3BFS_QPL][4];
#pragma unroll
      for (int r = 0; r < S3BFS_QPL; ++r) {
        const int cc[4] = {c[r].x, c[r].y, c[r].z, c[r].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool known = cc[j] < hub_lim && ((s_hub[cc[j] >> 5] >> (cc[j] & 31)) & 1u);
          vv[r][j] = pos[r] + j >= wp0[r] && pos[r] + j < wp1[r] && !known && in_range(p, cc[j], p.n, 14);
          lv[r][j] = vv[r][j] ? ld_level(level + cc[j]) : 0;
        }
      }
#pragma unroll
      for (int r = 0; r < S3BFS_QPL; ++r) {
        const int cc[4] = {c[r].x, c[r].y, c[r].z, c[r].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool k = vv[r][j] && lv[r][j] < 0;
          if (k) {
            st_relaxed(level + cc[j], lnext);
            st_relaxed(parent + cc[j], wu[r]);
          }
          cnt = emit(out, cnt, k, cc[j], wu[r], lane);
#if S3BFS_CHECKED
          // a chunk emits at most one candidate per edge of its region (the
          // buffer's 32 spare pairs absorb the slot that would pass it)
          if (!in_range(p, cnt, e_end - e_begin + 1, 15)) return e_end - e_begin;
#endif
        }
      }
    }
    i = i_next;
    e = tile_end;
  }
  return cnt;
}

// ---------------------------------------------------------------------------
// COMPACT: dedup, then a single-pass look-back scan over the CTAs of a level
// ---------------------------------------------------------------------------

// Direction of the next level of a direction-optimising traversal (Beamer,
// Asanovic and Patterson, SC 2012; the paper's conclusion names bottom-up
// steps as compatible with S3BFS).  With m_u = nnz - cum, the degree sum of
// the vertices still unvisited once the next frontier is known: a top-down
// traversal turns bottom-up when the next frontier's edges exceed m_u / alpha
// -- and, on a GPU where a bottom-up test costs about what a top-down one
// does, also gamma times the unvisited vertices of degree > 0 (each of which
// a bottom-up level visits; gamma = 0 drops this test); a bottom-up one
// turns back when the frontier shrinks below n / beta.
__device__ __forceinline__ int next_direction(const Params& p, int dir_l, long long n_l, long long n_next,
                                              long long e_next, long long cum, long long vcum) {
  if (!p.direction || n_next <= 0) return 0;
  const long long m_u = (long long)p.nnz - cum;
  const long long n_u = (long long)p.n_live - vcum;
  if (dir_l == 0) return (e_next * p.alpha > m_u && e_next > (long long)p.gamma * n_u) ? 1 : 0;
  return (n_next * p.beta < (long long)p.n && n_next < n_l) ? 0 : 1;
}

// Dedup (Fig. 1, owner check) and linearisation (Sizes prefix sum) of the candidates of one
// CTA's chunks, plus the degree gather and exclusive scan of the next frontier
// (Fig. 1's degree gather and EdgeSum of the next level).  Called by every thread of a CTA that holds
// at least one of the level's P_l chunks; warps without a chunk pass cnt = 0.
//
// Pass 1 (per warp): candidates 128 at a time (S3BFS_CR per lane), all loads
// in flight together; keep (v, u) iff parent[v] == u.  Survivors of the last
// batch stay in registers, earlier batches are stashed in place (kept index <=
// candidate index) as (v, row start) in cand with their degree prefix in aux.
// Scan: the CTA's aggregate (kept count, kept degree sum, candidates) is
// published with a release store; every CTA then sums the aggregates of all
// CTAs before it (256 at a time, no chain of inclusive prefixes to wait for)
// and adds its warps' offsets.  Pass 2 writes the survivors at their slots of
// the next frontier F / RS / EX.  The CTA holding chunk P_l - 1 publishes the
// next level's n and e.  Returns false (in every thread) if a wait ran out.
constexpr int kCompactR = S3BFS_CR;

// b: rank of this CTA among the CTAs that hold the level's chunks (the scan
// runs over ranks 0 .. (P_l - 1) / W).  work: neighbour entries this warp
// examined in the level (summed into the next level's control block).
// s_next (optional, shared memory): the publishing thread also leaves the
// next level's control block there (n = -1 when it raised an error), for a
// CTA that runs the next level alone.
#ifndef S3BFS_COMPACT_QUAL
#define S3BFS_COMPACT_QUAL
#endif
template <int W>  // warps per CTA
__device__ S3BFS_COMPACT_QUAL bool compact_cta(const Params& p, int l, int par, int P_l, int2* cand, int* aux, int cnt, int b,
                            int work, LevelCtrl* s_next = nullptr) {
  __shared__ int sK[W], sD[W], sC[W], sW[W];
  __shared__ int sRed[4][W];
  __shared__ int sPre[4];
  const int lane = threadIdx.x & (kWarp - 1);
  const int wib = threadIdx.x >> 5;
  const int np = par ^ 1;
  int* Fn = np ? p.F[1] : p.F[0];
  int* RSn = np ? p.RS[1] : p.RS[0];
  int* EXn = np ? p.EX[1] : p.EX[0];
  const unsigned lt = (1u << lane) - 1u;
#if S3BFS_CHECKED
  // vertices of levels <= l (read before the publishing thread rewrites s_next)
  const int vbase = p.fdump ? (s_next ? s_next->vcum : ld_relaxed(&p.st->ctrl[par].vcum)) : 0;
#endif

  // ---- pass 1
  int K = 0, D = 0, K_stash = 0;
  int v[kCompactR], rs[kCompactR], idx[kCompactR], dpre[kCompactR];
  bool keep[kCompactR];
#pragma unroll
  for (int r = 0; r < kCompactR; ++r) keep[r] = false;
  for (int base = 0; base < cnt; base += kWarp * kCompactR) {
    int2 pr[kCompactR];
    int pv[kCompactR], re[kCompactR];
#pragma unroll
    for (int r = 0; r < kCompactR; ++r) {
      const int j = base + r * kWarp + lane;
      pr[r] = j < cnt ? ld_cg2(cand + j) : make_int2(0, -2);
    }
#pragma unroll
    for (int r = 0; r < kCompactR; ++r)
      pv[r] = pr[r].y != -2 && in_range(p, pr[r].x, p.n, 20) ? ld_relaxed_nb(p.parent + pr[r].x) : -3;
#pragma unroll
    for (int r = 0; r < kCompactR; ++r) {
      keep[r] = pv[r] == pr[r].y;
      v[r] = pr[r].x;
      rs[r] = keep[r] ? __ldg(p.row_ptr + v[r]) : 0;
      re[r] = keep[r] ? __ldg(p.row_ptr + v[r] + 1) : 0;
    }
    K_stash = K;
#pragma unroll
    for (int r = 0; r < kCompactR; ++r) {
      const int deg = re[r] - rs[r];
      const unsigned m = __ballot_sync(kFull, keep[r]);
      const int incl = warp_incl_scan(deg, lane);
      idx[r] = K + __popc(m & lt);
      dpre[r] = D + incl - deg;
      K += __popc(m);
      D += __shfl_sync(kFull, incl, kWarp - 1);
    }
    if (base + kWarp * kCompactR < cnt) {
#pragma unroll
      for (int r = 0; r < kCompactR; ++r)
        if (keep[r]) {
          cand[idx[r]] = make_int2(v[r], rs[r]);
          aux[idx[r]] = dpre[r];
        }
    }
  }
  if (lane == 0) {
    sK[wib] = K;
    sD[wib] = D;
    sC[wib] = cnt;
    sW[wib] = work;
  }
  __syncthreads();

  // ---- scan over the CTAs of this level
  ChunkStatus* S = p.status;
  const unsigned long long ep = (unsigned long long)((unsigned)(l + 1) & kEpochMask) << 32;
  if (threadIdx.x == 0) {
    int Kc = 0, Dc = 0, Cc = 0, Wc = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      Kc += sK[w];
      Dc += sD[w];
      Cc += sC[w];
      Wc += sW[w];
    }
    S[b].agg_deg = Dc;
    S[b].agg_cand = Cc;
    S[b].agg_work = Wc;
    st_release64(&S[b].word, (kFlagAgg << 62) | ep | (unsigned)Kc);
  }
  int kk = 0, dd = 0, cc = 0, ww = 0;
  bool ok = in_range(p, b, p.max_chunks, 21);
  const long long t0 = global_ns();
  for (int j = threadIdx.x; j < b && ok; j += blockDim.x) {
    int it = 0;
    unsigned long long w;
    while (true) {
      w = ld_acquire64(&S[j].word);
      if ((unsigned)((w >> 32) & kEpochMask) == ((unsigned)(l + 1) & kEpochMask) && (w >> 62) != 0) break;
      if (ld_relaxed(&p.st->err) != 0) {
        ok = false;
        break;
      }
      if (++it > kSpinIters || global_ns() - t0 > p.spin_ns) {
        set_err(p, BFS_E_TIMEOUT, 3);
        ok = false;
        break;
      }
      if (it > 32) __nanosleep(32);
    }
    if (ok) {
      kk += (int)(unsigned)(w & 0xffffffffull);
      dd += ld_relaxed(&S[j].agg_deg);
      cc += ld_relaxed(&S[j].agg_cand);
      ww += ld_relaxed(&S[j].agg_work);
    }
  }
  kk = __reduce_add_sync(kFull, kk);
  dd = __reduce_add_sync(kFull, dd);
  cc = __reduce_add_sync(kFull, cc);
  ww = __reduce_add_sync(kFull, ww);
  if (lane == 0) {
    sRed[0][wib] = kk;
    sRed[1][wib] = dd;
    sRed[2][wib] = cc;
    sRed[3][wib] = ww;
  }
  ok = __syncthreads_and(ok);
  if (!ok) return false;
  if (threadIdx.x == 0) {
    int a = 0, d = 0, c = 0, x = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      a += sRed[0][w];
      d += sRed[1][w];
      c += sRed[2][w];
      x += sRed[3][w];
    }
    sPre[0] = a;
    sPre[1] = d;
    sPre[2] = c;
    sPre[3] = x;
  }
  __syncthreads();
  int Kx = sPre[0], Dx = sPre[1];
  for (int w = 0; w < wib; ++w) {
    Kx += sK[w];
    Dx += sD[w];
  }

  // ---- pass 2: stashed batches (a copy with offsets), then the register batch
  for (int base = 0; base < K_stash; base += kWarp * kCompactR) {
    int2 sv[kCompactR];
    int sd[kCompactR];
#pragma unroll
    for (int r = 0; r < kCompactR; ++r) {
      const int i = base + r * kWarp + lane;
      if (i < K_stash) {
        sv[r] = ld_cg2(cand + i);
        sd[r] = ld_cg(aux + i);
      }
    }
#pragma unroll
    for (int r = 0; r < kCompactR; ++r) {
      const int i = base + r * kWarp + lane;
      const int pos = Kx + i;
      if (i < K_stash && pos < p.n) {
        Fn[pos] = sv[r].x;
        RSn[pos] = sv[r].y;
        EXn[pos] = Dx + sd[r];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kCompactR; ++r) {
    const int pos = Kx + idx[r];
    if (keep[r] && pos < p.n) {
      Fn[pos] = v[r];
      RSn[pos] = rs[r];
      EXn[pos] = Dx + dpre[r];
    }
  }
#if S3BFS_CHECKED
  if (p.fdump) {
    // the next frontier in level order: after the vertices of levels <= l
    for (int base = 0; base < K_stash; base += kWarp * kCompactR)
#pragma unroll
      for (int r = 0; r < kCompactR; ++r) {
        const int i = base + r * kWarp + lane;
        if (i < K_stash && in_range(p, (long long)vbase + Kx + i, p.n, 22)) p.fdump[vbase + Kx + i] = ld_cg2(cand + i).x;
      }
#pragma unroll
    for (int r = 0; r < kCompactR; ++r)
      if (keep[r] && in_range(p, (long long)vbase + Kx + idx[r], p.n, 23)) p.fdump[vbase + Kx + idx[r]] = v[r];
  }
#endif
  if (b == (P_l - 1) / W && threadIdx.x == 0) {
    long long n_next = sPre[0], e_next = sPre[1], c_l = sPre[2], w_l = sPre[3];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      n_next += sK[w];
      e_next += sD[w];
      c_l += sC[w];
      w_l += sW[w];
    }
    const LevelCtrl cur = s_next ? *s_next : LevelCtrl{ld_relaxed(&p.st->ctrl[par].n), 0, 0,
                                                         ld_relaxed(&p.st->ctrl[par].cum),
                                                         ld_relaxed(&p.st->ctrl[par].dir), 0, 0,
                                                         ld_relaxed(&p.st->ctrl[par].vcum)};
    const long long cum = (long long)cur.cum + e_next;
    const long long vcum = (long long)cur.vcum + n_next;
    if (n_next > p.n || e_next > p.nnz || e_next < 0 || cum > p.nnz) {
      set_err(p, BFS_E_MULTIGRAPH, 4);
      if (s_next) s_next->n = -1;
    } else {
      EXn[n_next] = (int)e_next;
      const int dir_l = cur.dir;
      const int dir_next = next_direction(p, dir_l, cur.n, n_next, e_next, cum, vcum);
      LevelCtrl* c = &p.st->ctrl[np];
      st_relaxed(&c->n, (int)n_next);
      st_relaxed(&c->e, (int)e_next);
      st_relaxed(&c->c, (int)c_l);
      st_relaxed(&c->cum, (int)cum);
      st_relaxed(&c->dir, dir_next);
      st_relaxed(&c->fb, dir_l);
      st_relaxed(&c->w, (int)w_l);
      st_relaxed(&c->vcum, (int)vcum);
      if (s_next)
        *s_next = LevelCtrl{(int)n_next, (int)e_next, (int)c_l, (int)cum, dir_next, dir_l, (int)w_l, (int)vcum};
      if (l < p.lvl_cap) {
        p.lvl[(long long)l * kLevelFields + 2] = (int)c_l;
        p.lvl[(long long)l * kLevelFields + 8] = (int)w_l;
      }
    }
  }
  return true;
}

// Bits of vertices [0, 32 * words) from the level array: bit v set iff
// level[v] == l, or iff level[v] >= 0 (visited) when l < 0.  A warp writes
// four words at a time (four coalesced loads in flight per lane, one ballot
// per word); words is a multiple of 4.  Every word is written.
__device__ __forceinline__ void level_bits(const Params& p, int l, int words, uint32_t* out, int gw, int P) {
  const int lane = threadIdx.x & (kWarp - 1);
  for (int q = gw; q < (words >> 2); q += P) {
    int lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = (q << 7) + (j << 5) + lane;
      lv[j] = v < p.n ? ld_relaxed_nb(p.level + v) : -1;
    }
    unsigned m[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) m[j] = __ballot_sync(kFull, l >= 0 ? lv[j] == l : lv[j] >= 0);
    if (lane < 4) out[(q << 2) + lane] = lane == 0 ? m[0] : lane == 1 ? m[1] : lane == 2 ? m[2] : m[3];
  }
}

// Visited bits of vertices [0, hub_n), from the level array after a level's
// explore (all its level stores are visible).
__device__ __forceinline__ void build_hub_bits(const Params& p, int gw, int P) {
  level_bits(p, -1, p.hub_n >> 5, p.hub_bits, gw, P);
}

// Copies the visited bits into shared memory (whole CTA); returns hub_n.
__device__ __forceinline__ int load_hub_bits(const Params& p, uint32_t* s_hub) {
  const int q = p.hub_n >> 7;
  const uint4* src = reinterpret_cast<const uint4*>(p.hub_bits);
  uint4* dst = reinterpret_cast<uint4*>(s_hub);
  for (int i = threadIdx.x; i < q; i += blockDim.x) dst[i] = ld_cg4u(src + i);
  __syncthreads();
  return p.hub_n;
}

// ---------------------------------------------------------------------------
// BOTTOM-UP levels of a direction-optimising traversal (symmetric graphs)
// ---------------------------------------------------------------------------

// Entries of its row a lane tests by itself; a longer row without a parent in
// them is then scanned by the whole warp, 32 entries a step.
#ifndef S3BFS_BU_LANE
#define S3BFS_BU_LANE 32
#endif
constexpr int kBuLane = S3BFS_BU_LANE;

// frontier-bitmap word: written before the last grid barrier (acquire), read
// through L1
__device__ __forceinline__ unsigned ld_bits(const uint32_t* p) {
  unsigned v;
  asm volatile("ld.global.ca.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
// Is u in the frontier of level l?  With S3BFS_BU_BITMAP the test reads the
// frontier bitmap (n bits, rebuilt from the level array around every
// bottom-up level); without, the level array itself (level[u] == l: no
// rebuild passes and no grid barrier for them, one 32-byte sector per test
// instead of one per 256 vertices).
#ifndef S3BFS_BU_BITMAP
#define S3BFS_BU_BITMAP 0
#endif
__device__ __forceinline__ bool in_frontier(const Params& p, const uint32_t* fb, int l, int u) {
  if (!in_range(p, u, p.n, 32)) return false;
#if S3BFS_BU_BITMAP
  (void)p;
  (void)l;
  return (ld_bits(fb + (u >> 5)) >> (u & 31)) & 1u;
#else
  (void)fb;
  return ld_level(p.level + u) == l;
#endif
}

// Frontier bitmap of level l from the level array: bit v set iff level[v] == l.
__device__ __forceinline__ void build_frontier_bits(const Params& p, int l, uint32_t* fb, int gw, int P) {
  level_bits(p, l, p.nwords, fb, gw, P);
}

// Vertices per lane in a bottom-up scan (independent parent searches in
// flight together).
#ifndef S3BFS_BU_V
#define S3BFS_BU_V 2
#endif
constexpr int kBuV = S3BFS_BU_V;
// entries tested in the first step of a row (1 to 4)
#ifndef S3BFS_BU_FIRST
#define S3BFS_BU_FIRST 1
#endif
constexpr int kBuFirst = S3BFS_BU_FIRST;

// Parent search of kBuV unvisited vertices per lane (slot j active if act[j];
// row entries [k[j], re[j]) in CSR order).  Each lane tests the first kBuLane
// entries of its rows, four a step per row; the rows still without a parent
// after that are scanned by the whole warp in turn, 32 entries a step.  The
// first neighbour in the frontier (bit set in fb) is the parent.  Warp-wide.
__device__ __forceinline__ void bu_search(const Params& p, const uint32_t* fb, int l, const bool* act, int* k,
                                          const int* re, bool* found, int* pu, int* wk) {
  const int lane = threadIdx.x & (kWarp - 1);
  int lim[kBuV];
  bool go[kBuV];
  bool any = false;
#pragma unroll
  for (int s = 0; s < kBuV; ++s) {
    found[s] = false;
    pu[s] = 0;
    lim[s] = act[s] ? min(re[s], k[s] + kBuLane) : k[s];
    go[s] = act[s] && k[s] < lim[s];
    any |= go[s];
  }
  // the first step tests kBuFirst entries (the row's first entries are its
  // highest-degree neighbours on a renumbered graph, the likeliest to be in
  // the frontier); every later step four
  int seen = 0, width = kBuFirst;
  while (__any_sync(kFull, any)) {
    int c[kBuV][4];
#pragma unroll
    for (int s = 0; s < kBuV; ++s)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        c[s][j] = go[s] && j < width && k[s] + j < lim[s] ? __ldg(p.col_idx + k[s] + j) : -1;
    bool h[kBuV][4];
#pragma unroll
    for (int s = 0; s < kBuV; ++s)
#pragma unroll
      for (int j = 0; j < 4; ++j) h[s][j] = c[s][j] >= 0 && in_frontier(p, fb, l, c[s][j]);
    any = false;
#pragma unroll
    for (int s = 0; s < kBuV; ++s) {
      if (go[s]) {
        int taken = min(width, lim[s] - k[s]);
#pragma unroll
        for (int j = 3; j >= 0; --j)
          if (h[s][j]) {
            found[s] = true;
            pu[s] = c[s][j];
            taken = j + 1;
          }
        seen += taken;
        k[s] = min(k[s] + width, lim[s]);  // the warp phase resumes exactly at lim
        go[s] = !found[s] && k[s] < lim[s];
      }
      any |= go[s];
    }
    width = 4;
  }
#pragma unroll
  for (int s = 0; s < kBuV; ++s) {
    unsigned hm = __ballot_sync(kFull, act[s] && !found[s] && k[s] < re[s]);
    while (hm) {
      const int j = __ffs(hm) - 1;
      hm &= hm - 1;
      const int hb = __shfl_sync(kFull, k[s], j), he = __shfl_sync(kFull, re[s], j);
      int hit = -1, n_seen = 0;
      for (int base = hb; base < he; base += kWarp) {
        const int e = base + lane;
        const int c = e < he ? __ldg(p.col_idx + e) : -1;
        const unsigned m = __ballot_sync(kFull, c >= 0 && in_frontier(p, fb, l, c));
        if (m) {
          const int first = __ffs(m) - 1;
          hit = __shfl_sync(kFull, c, first);
          n_seen += first + 1;
          break;
        }
        n_seen += min(kWarp, he - base);
      }
      if (lane == j) {
        seen += n_seen;
        if (hit >= 0) {
          found[s] = true;
          pu[s] = hit;
        }
      }
    }
  }
  *wk += seen;
}

// A bottom-up level that follows a top-down one starts by listing, per warp,
// the unvisited vertices of degree > 0 among the 128-vertex groups gw, gw +
// P, ... (level and row bounds of four 32-vertex words in flight per lane).
// Each listed vertex first tests its first neighbour: most find their parent
// there (the highest-degree neighbour on a renumbered graph), are written and
// emitted at once (*found candidates to out, *work entries examined) and
// never enter the list.  Returns the list length (at most 128 per group).
__device__ inline int bu_unvisited(const Params& p, int l, const uint32_t* fb, int gw, int P, int* ulist, int2* out,
                                   int* found, int* work) {
  const int lane = threadIdx.x & (kWarp - 1);
  const unsigned lt = (1u << lane) - 1u;
  int cnt = 0, nf = 0, wk = 0;
  for (int q = gw; q < p.bu_groups; q += P) {
    int lv[4], rs[4], re[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = (q << 7) + (j << 5) + lane;
      lv[j] = v < p.n ? ld_relaxed_nb(p.level + v) : 0;
      rs[j] = v <= p.n ? __ldg(p.row_ptr + v) : 0;  // row_ptr[n] ends the last row
      re[j] = __shfl_down_sync(kFull, rs[j], 1);
      if (lane == kWarp - 1) re[j] = v < p.n ? __ldg(p.row_ptr + v + 1) : 0;
    }
    bool unv[4];
    int c0[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = (q << 7) + (j << 5) + lane;
      unv[j] = v < p.n && lv[j] < 0 && re[j] > rs[j];
      c0[j] = unv[j] ? __ldg(p.col_idx + rs[j]) : -1;
      if (c0[j] >= 0 && !in_range(p, c0[j], p.n, 30)) c0[j] = -1;
    }
    bool hit[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) hit[j] = c0[j] >= 0 && in_frontier(p, fb, l, c0[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = (q << 7) + (j << 5) + lane;
      wk += unv[j] ? 1 : 0;
      if (hit[j]) {
        p.level[v] = l + 1;
        p.parent[v] = c0[j];
      }
      const unsigned fm = __ballot_sync(kFull, hit[j]);
      if (hit[j]) out[nf + __popc(fm & lt)] = make_int2(v, c0[j]);
      nf += __popc(fm);
      const bool keep = unv[j] && !hit[j];
      const unsigned km = __ballot_sync(kFull, keep);
      if (keep) ulist[cnt + __popc(km & lt)] = v;
      cnt += __popc(km);
    }
  }
  *found = nf;
  *work = wk;
  return cnt;
}

// One warp's share of a bottom-up level l: its list of unvisited vertices
// (kBuV * 32 at a time).  Every vertex looks for a parent in the frontier of
// level l; a vertex found gets level l + 1 and its parent from its own lane
// (no other lane writes it, so the candidates (v, parent) emitted here all
// survive the compaction's dedup); the others stay in the list, compacted in
// place (a kept entry never lands past one not yet read).  Returns the
// candidates written to out; *work = neighbour entries examined (warp total).
// skip: the first entry of every row was tested already (by bu_unvisited).
__device__ inline int bu_scan(const Params& p, int l, const uint32_t* fb, int gw, int total, int* ulist, int2* out,
                              int* work, int skip) {
  const int lane = threadIdx.x & (kWarp - 1);
  const unsigned lt = (1u << lane) - 1u;
  int cnt = 0, kept = 0, wk = 0;
  for (int b = 0; b < total; b += kWarp * kBuV) {
    bool act[kBuV];
    int v[kBuV], k[kBuV], re[kBuV];
#pragma unroll
    for (int s = 0; s < kBuV; ++s) {
      const int i = b + s * kWarp + lane;
      act[s] = i < total;
      v[s] = act[s] ? ld_relaxed_nb(ulist + i) : 0;
      if (act[s] && !in_range(p, v[s], p.n, 31)) act[s] = false;
    }
#pragma unroll
    for (int s = 0; s < kBuV; ++s) {
      k[s] = act[s] ? __ldg(p.row_ptr + v[s]) + skip : 0;
      re[s] = act[s] ? __ldg(p.row_ptr + v[s] + 1) : 0;
    }
    bool found[kBuV];
    int pu[kBuV];
    bu_search(p, fb, l, act, k, re, found, pu, &wk);
#pragma unroll
    for (int s = 0; s < kBuV; ++s) {
      if (found[s]) {
        p.level[v[s]] = l + 1;
        p.parent[v[s]] = pu[s];
      }
      const unsigned fm = __ballot_sync(kFull, found[s]);
      if (found[s]) out[cnt + __popc(fm & lt)] = make_int2(v[s], pu[s]);
      cnt += __popc(fm);
      const bool keep = act[s] && !found[s];
      const unsigned km = __ballot_sync(kFull, keep);
      if (keep) ulist[kept + __popc(km & lt)] = v[s];
      kept += __popc(km);
    }
  }
  if (lane == 0) p.ulist_cnt[gw] = kept;
  *work = __reduce_add_sync(kFull, wk);
  return cnt;
}

__device__ __forceinline__ void publish_empty_next(const Params& p, int par) {
  LevelCtrl* c = &p.st->ctrl[par ^ 1];
  st_relaxed(&c->n, 0);
  st_relaxed(&c->e, 0);
  st_relaxed(&c->c, 0);
  st_relaxed(&c->dir, 0);
  st_relaxed(&c->fb, 0);
  st_relaxed(&c->w, 0);
}

__device__ __forceinline__ void record_level(const Params& p, int l, int n_l, int e_l, int P_l, int dir = 0) {
  if (l < p.lvl_cap) {
    int* r = p.lvl + (long long)l * kLevelFields;
    r[0] = n_l;
    r[1] = e_l;
    r[2] = 0;
    r[3] = P_l;
    r[4] = 0;
    r[5] = 0;
    r[6] = 0;
    r[7] = dir;
    r[8] = 0;
  }
}

// a0 (Fig. 1, initialisation): level = parent = -1 except level[s] = 0, parent[s] =
// s; F_0 = [s] with its row start and degree; clear the scan and barrier
// state (ctas arrival words; none if 0) and the visited bits.  Grid-stride.
__device__ __forceinline__ void init_traversal(const Params& p, int ctas) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int s = p.src;
  // entries to clear (parents are cleared only where they are not lazy, and
  // there level_n is n)
  const int n = (p.parent_lazy && p.level_n > 0 && p.level_n < p.n) ? p.level_n : p.n;
  if (tid == 0 && s >= n) p.level[s] = 0;  // an isolated source past the cleared part
  const bool vec = ((reinterpret_cast<uintptr_t>(p.level) | reinterpret_cast<uintptr_t>(p.parent)) & 15) == 0;
  if (vec) {
    int4* L4 = reinterpret_cast<int4*>(p.level);
    int4* P4 = reinterpret_cast<int4*>(p.parent);
    const long long n4 = n >> 2;
    for (long long i = tid; i < n4; i += stride) {
      int4 lv = make_int4(-1, -1, -1, -1), pv = make_int4(-1, -1, -1, -1);
      const long long b = i << 2;
      if (s >= b && s < b + 4) {
        const int o = (int)(s - b);
        if (o == 0) { lv.x = 0; pv.x = s; }
        if (o == 1) { lv.y = 0; pv.y = s; }
        if (o == 2) { lv.z = 0; pv.z = s; }
        if (o == 3) { lv.w = 0; pv.w = s; }
      }
      L4[i] = lv;
      if (!p.parent_lazy) P4[i] = pv;
    }
    for (long long v = (n4 << 2) + tid; v < n; v += stride) {
      p.level[v] = v == s ? 0 : -1;
      if (!p.parent_lazy) p.parent[v] = v == s ? s : -1;
    }
  } else {
    for (long long v = tid; v < n; v += stride) {
      p.level[v] = v == s ? 0 : -1;
      if (!p.parent_lazy) p.parent[v] = v == s ? s : -1;
    }
  }
  if (p.parent_lazy && tid == 0) p.parent[s] = s;
  for (long long i = tid; i < p.max_chunks; i += stride) p.status[i].word = 0ull;
  for (long long i = tid; i < ((ctas + 3) & ~3); i += stride) p.bar_arrive[i] = 0;
  for (long long i = tid; i < (p.hub_n >> 5); i += stride) p.hub_bits[i] = 0u;
  if (tid == 0) {
    const int rs = p.row_ptr[s], deg = p.row_ptr[s + 1] - rs;
#if S3BFS_CHECKED
    if (p.fdump) p.fdump[0] = s;
#endif
    p.F[0][0] = s;
    p.RS[0][0] = rs;
#if S3BFS_CHECKED
    if (p.debug_flags & BFS_DEBUG_CHECK_INJECT) p.RS[0][0] = p.nnz + 8;  // caught by range check 13
#endif
    p.EX[0][0] = 0;
    p.EX[0][1] = deg;
    DevState* st = p.st;
    LevelCtrl c0 = {1, deg, 0, deg, 0, 0, 0, 1};
    LevelCtrl c1 = {0, 0, 0, 0, 0, 0, 0, 0};
    st->ctrl[0] = c0;
    st->ctrl[1] = c1;
    st->err = 0;
    st->err_where = 0;
    st->num_levels = 0;
    st->bar_release = 0;
    st->reached = st->edges = st->cands = 0;
    st->progress = 0;
    st->resume_level = 0;
    st->work = 0;
  }
}

// Internal ids i >= n_kept are isolated vertices whose level entries the
// traversal never touched: -1, except the source s (level 0, its own parent).
__device__ __forceinline__ void finalize_outputs(int32_t n, const int32_t* inv, const int32_t* perm,
                                                 const int32_t* level, const int32_t* parent, int32_t* level_out,
                                                 int32_t* parent_out, int32_t n_kept, int32_t s) {
  // four vertices a thread per step, their loads in flight together (the
  // chain inv -> level, parent -> perm is latency-bound)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; v0 < n; v0 += 4 * stride) {
    int i[4], lv[4], q[4], pp[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { const long long v = v0 + k * stride; i[k] = v < n ? __ldg(inv + v) : 0; }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long v = v0 + k * stride;
      const bool kept = v < n && i[k] < n_kept;
      lv[k] = kept ? level[i[k]] : (v < n && i[k] == s ? 0 : -1);
      // an unreached vertex's parent entry may never have been written
      q[k] = (kept && parent_out) ? parent[i[k]] : i[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) pp[k] = (lv[k] >= 0 && parent_out) ? __ldg(perm + q[k]) : -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long v = v0 + k * stride;
      if (v < n) {
        level_out[v] = lv[k];
        if (parent_out) parent_out[v] = pp[k];
      }
    }
  }
}

}  // namespace s3bfs
