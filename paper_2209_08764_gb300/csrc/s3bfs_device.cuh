// S3BFS level step on sm_103a: device code.
//
// One level of Parallel-BFS (Fig. 1, lines 10-29) runs as two phases separated
// by a grid-wide barrier:
//
//   EXPLORE  (lines 16-18)  the level's e_l edges are split into P_l chunks of
//            C_l = ceil(e_l / P_l) consecutive edges, one chunk per warp, with
//            P_l = min(P, ceil(e_l / grain)) (line 16; grain = 1 is the paper's
//            formula).  A warp finds its start (frontier entry, edge offset) by
//            a search on the exclusive degree scan EX (line 17), then walks its
//            edges: for an edge (u, v) with level[v] == -1 it stores
//            level[v] = l + 1 and parent[v] = u with plain (relaxed, non-RMW)
//            stores and emits the candidate pair (v, u) into its own region of
//            the candidate buffer (line 18; Algorithm paragraph).
//   COMPACT  (lines 19-29)  each warp re-reads parent[v] for its candidates and
//            keeps (v, u) iff parent[v] == u: the owner of v is the vertex
//            whose store to parent[v] landed last, so exactly one candidate
//            per newly reached v survives (lines 19-23 with the owner id taken
//            to be the parent vertex).  A single-pass decoupled look-back scan
//            over the chunks, in chunk order, gives every survivor its slot in
//            the next frontier (lines 24-29) and, in the same pass, the
//            exclusive prefix sum of the survivors' degrees, i.e. the next
//            level's degree gather and EdgeSum scan (lines 12-15).
//
// The next frontier is stored as three int32 arrays: F (vertex), RS (first CSR
// position of its row) and EX (exclusive degree prefix, with EX[n] = e).
// No atomic read-modify-write instruction is used anywhere: the paper's BFS
// "does not use locks and atomic-instructions" (Abstract).  Cross-warp
// ordering uses release/acquire stores and loads only.
#pragma once

#include <cstdint>

#include "s3bfs.h"

namespace s3bfs {

constexpr int kWarp = 32;
constexpr int kWarpsPerCta = 8;
constexpr int kThreads = kWarp * kWarpsPerCta;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kLevelFields = BFS_LEVEL_FIELDS;
// hard iteration cap of every spin-wait, on top of the time limit
constexpr int kSpinIters = 1 << 21;

constexpr unsigned long long kFlagAgg = 1ull;
constexpr unsigned long long kFlagIncl = 2ull;
constexpr unsigned kEpochMask = 0x3FFFFFFFu;

// Look-back state of one chunk: word = [63:62] flag, [61:32] epoch (level+1),
// [31:0] kept count.  The degree and candidate sums sit in separate slots for
// the aggregate and the inclusive prefix, written before the word is released.
struct alignas(32) ChunkStatus {
  unsigned long long word;
  int32_t agg_deg, agg_cand, incl_deg, incl_cand;
  int32_t pad[2];
};

struct LevelCtrl {
  int32_t n, e, c, pad;
};

// Device-resident control block of one traversal.
struct DevState {
  LevelCtrl ctrl[2];  // size n and edge count e of the frontier of level l, by parity of l
  int32_t err;        // 0 or a BFS_E_* code
  int32_t err_where;  // which wait or check failed
  int32_t num_levels;
  int32_t bar_release;
  long long reached, edges, cands;
};

struct Params {
  int32_t n, nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;  // padded: readable up to a multiple of 4 entries past nnz
  int32_t* level;
  int32_t* parent;
  int32_t* F[2];
  int32_t* RS[2];
  int32_t* EX[2];
  int2* cand;           // candidate pairs (v, u); chunk k owns [k*C_l, (k+1)*C_l)
  int32_t* cand_cnt;    // per chunk, for the launch-per-phase mode
  ChunkStatus* status;  // per chunk
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

__device__ __forceinline__ void set_err(const Params& p, int code, int where) {
  st_relaxed(&p.st->err_where, where);
  st_relaxed(&p.st->err, code);
}

__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const int t = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += t;
  }
  return x;
}

// P_l and C_l of a level (Fig. 1 line 16 with a grain; Algorithm paragraph:
// "(almost) equal division" of the e_l edges).  Shared by host and device.
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
// word; CTA 0 waits for all of them and releases one word everybody waits on.
// Every wait is bounded by the time limit and an iteration cap; on expiry the
// error word is set and all CTAs return false.  Also returns false, in every
// CTA, when any CTA raised an error before the barrier.
// ---------------------------------------------------------------------------
__device__ bool grid_sync(const Params& p, int epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool stall =
        (p.debug_flags & BFS_DEBUG_STALL_BARRIER) && epoch == 1 && blockIdx.x == gridDim.x - 1;
    __threadfence();
    if (!stall) st_relaxed(&p.bar_arrive[blockIdx.x], epoch);
  }
  if (blockIdx.x == 0) {
    bool ok = true;
    const long long t0 = global_ns();
    for (int j = threadIdx.x; j < (int)gridDim.x && ok; j += blockDim.x) {
      int it = 0;
      while (ld_relaxed(&p.bar_arrive[j]) < epoch) {
        if (ld_relaxed(&p.st->err) != 0) {
          ok = false;
          break;
        }
        if (++it > kSpinIters || global_ns() - t0 > p.spin_ns) {
          set_err(p, BFS_E_TIMEOUT, 1);
          ok = false;
          break;
        }
        if (it > 64) __nanosleep(100);
      }
    }
    ok = __syncthreads_and(ok);
    if (threadIdx.x == 0 && ok) {
      __threadfence();
      st_relaxed(&p.st->bar_release, epoch);
    }
  }
  if (threadIdx.x == 0) {
    int ok = 1, it = 0;
    const long long t0 = global_ns();
    while (ld_relaxed(&p.st->bar_release) < epoch) {
      if (ld_relaxed(&p.st->err) != 0) {
        ok = 0;
        break;
      }
      if (++it > kSpinIters || global_ns() - t0 > p.spin_ns) {
        set_err(p, BFS_E_TIMEOUT, 2);
        ok = 0;
        break;
      }
      if (it > 64) __nanosleep(64);
    }
    __threadfence();
    // one decision per CTA: an error raised before the barrier by any CTA
    // (a timeout, or a frontier larger than n) makes every CTA leave
    s_ok = ok && ld_relaxed(&p.st->err) == 0;
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
__device__ int explore_chunk(const Params& p, int l, int par, int n_l, int e_l, int e_begin, int e_end,
                             int2* out) {
  const int lane = threadIdx.x & (kWarp - 1);
  // (selects, not p.EX[par]: a runtime index into the parameter block would
  // copy it to local memory)
  const int* EX = par ? p.EX[1] : p.EX[0];
  const int* F = par ? p.F[1] : p.F[0];
  const int* RS = par ? p.RS[1] : p.RS[0];
  const int4* col4 = reinterpret_cast<const int4*>(p.col_idx);
  int* level = p.level;
  int* parent = p.parent;
  const int lnext = l + 1;

  // Find-StartExpPoint (line 17): the last frontier entry i with EX[i] <=
  // e_begin (upper bound minus one), by a 32-ary search -- every round the
  // lanes probe 32 evenly spaced entries of [lo, hi) and keep the last probe
  // that is still <= e_begin.  Invariant: EX[lo] <= e_begin < EX[hi].
  int lo = 0, hi = n_l;
  while (hi - lo > 1) {
    const int step = (hi - lo + kWarp - 1) / kWarp;
    const int idx = lo + lane * step;
    const bool le = idx < hi && ld_cg(EX + idx) <= e_begin;
    const unsigned m = __ballot_sync(kFull, le);
    const int J = 31 - __clz(m);
    lo += J * step;
    hi = min(lo + step, hi);
  }

  int i = lo;  // current frontier entry
  int e = e_begin;
  int cnt = 0;
  while (e < e_end) {
    // Stage a window of 32 frontier entries, one per lane: its first edge
    // EX[idx], the edge after its last EX[idx+1], its row start and vertex.
    const int idx = i + lane;
    const bool in = idx < n_l;
    const int ex_lo = in ? ld_cg(EX + idx) : e_l;
    int ex_hi = __shfl_down_sync(kFull, ex_lo, 1);
    if (lane == kWarp - 1) ex_hi = in ? ld_cg(EX + idx + 1) : e_l;
    const int rs = in ? ld_cg(RS + idx) : 0;
    const int u = in ? ld_cg(F + idx) : 0;
    const int tile_end = min(e_end, __shfl_sync(kFull, ex_hi, kWarp - 1));
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
    // Load-balanced walk: round r hands quad r*32+lane to this lane; its owner
    // entry w is the first lane whose quad range ends after it.
    for (int base = 0; base < Q; base += kWarp) {
      const int q = base + lane;
      int w = 0;
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) {
        const int t = __shfl_sync(kFull, qend, w + s - 1);
        if (t <= q) w += s;
      }
      const bool act = q < Q;
      const int wq0 = __shfl_sync(kFull, q0, w);
      const int wqoff = __shfl_sync(kFull, qoff, w);
      const int wp0 = __shfl_sync(kFull, p0, w);
      const int wp1 = __shfl_sync(kFull, p1, w);
      const int wu = __shfl_sync(kFull, u, w);
      const int qa = wq0 + (q - wqoff);
      int4 c = make_int4(0, 0, 0, 0);
      if (act) c = ld_nc4(col4 + qa);
      const int pos = qa << 2;
      const bool v0 = act && pos >= wp0 && pos < wp1;
      const bool v1 = act && pos + 1 >= wp0 && pos + 1 < wp1;
      const bool v2 = act && pos + 2 >= wp0 && pos + 2 < wp1;
      const bool v3 = act && pos + 3 >= wp0 && pos + 3 < wp1;
      int l0 = 0, l1 = 0, l2 = 0, l3 = 0;
      if (v0) l0 = ld_relaxed_nb(level + c.x);
      if (v1) l1 = ld_relaxed_nb(level + c.y);
      if (v2) l2 = ld_relaxed_nb(level + c.z);
      if (v3) l3 = ld_relaxed_nb(level + c.w);
      const bool k0 = v0 && l0 < 0;
      const bool k1 = v1 && l1 < 0;
      const bool k2 = v2 && l2 < 0;
      const bool k3 = v3 && l3 < 0;
      if (k0) { st_relaxed(level + c.x, lnext); st_relaxed(parent + c.x, wu); }
      if (k1) { st_relaxed(level + c.y, lnext); st_relaxed(parent + c.y, wu); }
      if (k2) { st_relaxed(level + c.z, lnext); st_relaxed(parent + c.z, wu); }
      if (k3) { st_relaxed(level + c.w, lnext); st_relaxed(parent + c.w, wu); }
      cnt = emit(out, cnt, k0, c.x, wu, lane);
      cnt = emit(out, cnt, k1, c.y, wu, lane);
      cnt = emit(out, cnt, k2, c.z, wu, lane);
      cnt = emit(out, cnt, k3, c.w, wu, lane);
    }
    // advance past the entries whose edges are all done
    i += __popc(__ballot_sync(kFull, in && ex_hi <= tile_end));
    e = tile_end;
  }
  return cnt;
}

// ---------------------------------------------------------------------------
// COMPACT: decoupled look-back over the chunks of one level
// ---------------------------------------------------------------------------

// Publishes chunk k's aggregate (kept count K, kept degree sum D, candidates
// C), accumulates the predecessors' values (32 at a time, stopping at the
// nearest inclusive prefix) and publishes k's inclusive prefix.
__device__ bool lookback(const Params& p, int k, int epoch, int K, int D, int C, int* Kx, int* Dx,
                         int* Cx) {
  const int lane = threadIdx.x & (kWarp - 1);
  ChunkStatus* S = p.status;
  const unsigned long long ep = (unsigned long long)((unsigned)epoch & kEpochMask) << 32;
  if (lane == 0) {
    if (k == 0) {
      S[0].incl_deg = D;
      S[0].incl_cand = C;
      st_release64(&S[0].word, (kFlagIncl << 62) | ep | (unsigned)K);
    } else {
      S[k].agg_deg = D;
      S[k].agg_cand = C;
      st_release64(&S[k].word, (kFlagAgg << 62) | ep | (unsigned)K);
    }
  }
  int kx = 0, dx = 0, cx = 0;
  if (k > 0) {
    int j = k - 1;
    const long long t0 = global_ns();
    while (true) {
      const int idx = j - lane;
      unsigned long long w = 0;
      bool ok = true;
      if (idx >= 0) {
        int it = 0;
        while (true) {
          w = ld_acquire64(&S[idx].word);
          if ((unsigned)((w >> 32) & kEpochMask) == ((unsigned)epoch & kEpochMask) && (w >> 62) != 0) break;
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
      }
      if (__any_sync(kFull, !ok)) return false;
      const unsigned long long flag = idx >= 0 ? (w >> 62) : 0ull;
      const unsigned incl = __ballot_sync(kFull, flag == kFlagIncl);
      const int stop = incl ? __ffs(incl) - 1 : kWarp - 1;
      int kk = 0, dd = 0, cc = 0;
      if (idx >= 0 && lane <= stop) {
        kk = (int)(unsigned)(w & 0xffffffffull);
        if (flag == kFlagIncl) {
          dd = ld_relaxed(&S[idx].incl_deg);
          cc = ld_relaxed(&S[idx].incl_cand);
        } else {
          dd = ld_relaxed(&S[idx].agg_deg);
          cc = ld_relaxed(&S[idx].agg_cand);
        }
      }
      kx += __reduce_add_sync(kFull, kk);
      dx += __reduce_add_sync(kFull, dd);
      cx += __reduce_add_sync(kFull, cc);
      if (incl) break;
      j -= kWarp;
    }
    if (lane == 0) {
      S[k].incl_deg = dx + D;
      S[k].incl_cand = cx + C;
      st_release64(&S[k].word, (kFlagIncl << 62) | ep | (unsigned)(kx + K));
    }
  }
  *Kx = kx;
  *Dx = dx;
  *Cx = cx;
  return true;
}

// Dedup (lines 19-23) and linearisation (lines 24-29) of chunk k's candidate
// pairs cand[0, cnt), plus the degree gather and exclusive scan of the next
// frontier (lines 12-15 of the next level).  The last chunk publishes the
// next level's n and e.  Returns false if a wait ran out.
__device__ bool compact_chunk(const Params& p, int l, int par, int k, int P_l, const int2* cand, int cnt) {
  const int lane = threadIdx.x & (kWarp - 1);
  const int np = par ^ 1;
  int* Fn = np ? p.F[1] : p.F[0];
  int* RSn = np ? p.RS[1] : p.RS[0];
  int* EXn = np ? p.EX[1] : p.EX[0];
  const unsigned lt = (1u << lane) - 1u;
  // pass 1: this chunk's survivors and their degree sum
  int K = 0, D = 0;
  for (int base = 0; base < cnt; base += kWarp) {
    const int j = base + lane;
    bool keep = false;
    int deg = 0;
    if (j < cnt) {
      const int2 pr = ld_cg2(cand + j);
      keep = ld_relaxed_nb(p.parent + pr.x) == pr.y;
      if (keep) deg = __ldg(p.row_ptr + pr.x + 1) - __ldg(p.row_ptr + pr.x);
    }
    K += __popc(__ballot_sync(kFull, keep));
    D += __reduce_add_sync(kFull, deg);
  }
  int Kx, Dx, Cx;
  if (!lookback(p, k, l + 1, K, D, cnt, &Kx, &Dx, &Cx)) return false;
  // pass 2: write the survivors at their global slots
  int kb = Kx, db = Dx;
  for (int base = 0; base < cnt; base += kWarp) {
    const int j = base + lane;
    bool keep = false;
    int deg = 0, rs = 0, v = 0;
    if (j < cnt) {
      const int2 pr = ld_cg2(cand + j);
      v = pr.x;
      keep = ld_relaxed_nb(p.parent + v) == pr.y;
      if (keep) {
        rs = __ldg(p.row_ptr + v);
        deg = __ldg(p.row_ptr + v + 1) - rs;
      }
    }
    const unsigned m = __ballot_sync(kFull, keep);
    const int dincl = warp_incl_scan(deg, lane);
    if (keep) {
      const int pos = kb + __popc(m & lt);
      if (pos < p.n) {
        Fn[pos] = v;
        RSn[pos] = rs;
        EXn[pos] = db + dincl - deg;
      }
    }
    kb += __popc(m);
    db += __shfl_sync(kFull, dincl, kWarp - 1);
  }
  if (k == P_l - 1 && lane == 0) {
    const long long n_next = (long long)Kx + K;
    const long long e_next = (long long)Dx + D;
    if (n_next > p.n || e_next > p.nnz) {
      set_err(p, BFS_E_MULTIGRAPH, 4);
    } else {
      EXn[n_next] = (int)e_next;
      st_relaxed(&p.st->ctrl[np].n, (int)n_next);
      st_relaxed(&p.st->ctrl[np].e, (int)e_next);
      st_relaxed(&p.st->ctrl[np].c, Cx + cnt);
      if (l < p.lvl_cap) p.lvl[(long long)l * kLevelFields + 2] = Cx + cnt;
    }
  }
  return true;
}

__device__ __forceinline__ void publish_empty_next(const Params& p, int par) {
  LevelCtrl* c = &p.st->ctrl[par ^ 1];
  st_relaxed(&c->n, 0);
  st_relaxed(&c->e, 0);
  st_relaxed(&c->c, 0);
}

__device__ __forceinline__ void record_level(const Params& p, int l, int n_l, int e_l, int P_l) {
  if (l < p.lvl_cap) {
    int* r = p.lvl + (long long)l * kLevelFields;
    r[0] = n_l;
    r[1] = e_l;
    r[2] = 0;
    r[3] = P_l;
    r[4] = 0;
  }
}

}  // namespace s3bfs
