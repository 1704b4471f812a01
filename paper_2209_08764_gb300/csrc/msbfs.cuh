// Multi-source BFS: up to 64 traversals of one graph in one launch, with a
// uint64 bitmask per vertex (bit i = traversal i).
//
// Every level pulls: a vertex v ORs the frontier masks of its neighbours,
// keeps the bits it has not seen yet, and those sources reach v at this
// level.  Only the thread (or warp) that owns v writes v's masks, so no atomic
// read-modify-write is needed, as in the single-source level step.  A new
// bit i also gives v's level for source i and, as its parent, the first
// neighbour whose frontier mask carries bit i.  Pulling needs in-edges, so the
// graph must be symmetric (every edge has its reverse).
//
// The distance definition is the same as for one source (Parallel-BFS returns
// d[0:n-1] per source; Fig. 1 header); the bitmask batching itself is not in
// the paper.
#pragma once

#include "s3bfs_device.cuh"

namespace s3bfs {

// vertices with more neighbours than kMsHeavy are handled by a whole warp,
// with more than kMsHuge by a whole CTA
constexpr int kMsHeavy = 128;
constexpr int kMsHuge = 8192;
constexpr int kMsUnroll = 8;  // neighbour masks in flight per thread (light vertices)
// dynamic shared memory of k_msbfs when parents are written: per warp, per
// source bit, per lane, the row offset (< kMsHeavy, one byte) of the first
// neighbour of the lane's light vertex that carried the bit
constexpr int kMsParentSmem = kWarpsPerCta * 64 * kWarp;
static_assert(kMsHeavy <= 256, "light-vertex parent offsets are stored as bytes");

struct MsParams {
  int32_t n, k;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  unsigned long long* seen;      // per vertex: sources that reached it
  unsigned long long* fr[2];     // per vertex: sources for which it is in the frontier, by level parity
  const int32_t* heavy;          // vertices of degree in (kMsHeavy, kMsHuge]
  int32_t n_heavy;
  const int32_t* huge;           // vertices of degree > kMsHuge
  int32_t n_huge;
  int32_t* levels_out;           // k x n, source-major, the caller's vertex ids
  int32_t* parents_out;          // k x n or null
  const int32_t* perm;           // internal -> caller id, or null
  const int32_t* inv;            // caller -> internal id, or null
  unsigned long long* block_or;  // [2][gridDim.x] new bits per CTA, by level parity
  unsigned long long* level_bits;  // [lvl_cap] sources with new vertices at each level
  long long* block_edges;          // [gridDim.x] neighbour entries read, per CTA (whole batch)
  int32_t lvl_cap;
  DevState* st;
  int32_t* bar_arrive;
  long long spin_ns;
  int32_t debug_flags;
  // 1: the outputs were not cleared; the kernel ends by writing -1 to every
  // (source, vertex) pair it did not reach (each entry written once).  0: the
  // host cleared them to -1 first (graphs with many isolated vertices, where
  // writing the missing pairs piecemeal costs more than one clearing pass)
  int32_t write_missing;
};

__device__ __forceinline__ unsigned long long ld_cg64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.global.cg.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
  const unsigned lo = __reduce_or_sync(kFull, (unsigned)x);
  const unsigned hi = __reduce_or_sync(kFull, (unsigned)(x >> 32));
  return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long warp_or64_masked(unsigned long long x, unsigned mask) {
  const unsigned lo = __reduce_or_sync(mask, (unsigned)x);
  const unsigned hi = __reduce_or_sync(mask, (unsigned)(x >> 32));
  return ((unsigned long long)hi << 32) | lo;
}

// exclusive OR prefix over the lanes (lane order)
__device__ __forceinline__ unsigned long long warp_excl_or64(unsigned long long x, int lane) {
  unsigned long long v = x;
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v |= t;
  }
  const unsigned long long e = __shfl_up_sync(kFull, v, 1);
  return lane == 0 ? 0ull : e;
}

__device__ __forceinline__ int out_id(const MsParams& p, int v) { return p.perm ? __ldg(p.perm + v) : v; }

__device__ __forceinline__ void write_bits(const MsParams& p, unsigned long long bits, int V, int value,
                                           int32_t* out) {
  while (bits) {
    const int i = __ffsll((long long)bits) - 1;
    bits &= bits - 1;
    out[(long long)i * p.n + V] = value;
  }
}

// One launch for the whole batch; one grid barrier per level.
__global__ void __launch_bounds__(kThreads, 1) k_msbfs(MsParams p) {
  extern __shared__ uint8_t ms_dyn[];  // kMsParentSmem bytes when parents_out is set, else none
  __shared__ unsigned long long s_or[kWarpsPerCta];
  __shared__ unsigned long long s_any;
  __shared__ long long s_edges[kWarpsPerCta];
  long long my_edges = 0;
  const int lane = threadIdx.x & (kWarp - 1);
  const int wib = threadIdx.x >> 5;
  init_cta_err();
  uint8_t* s_off = ms_dyn + wib * 64 * kWarp;  // [source bit][lane]
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const int gw = (int)(tid >> 5);
  const int nwarps = (int)(nthreads >> 5);
  const unsigned long long full = p.k >= 64 ? ~0ull : ((1ull << p.k) - 1ull);
  const int* rp = p.row_ptr;
  const int* ci = p.col_idx;
  int l = 0, bar = 0;
  bool finished = false;  // the loop ended with no source advancing (not on an error)
  // sources with a non-empty frontier at this level: the only bits a vertex
  // can gain now.  A vertex stops pulling once it holds all of them (and
  // skips its row when it already did), the early exit of multi-source BFS.
  unsigned long long active = full;
  while (true) {
    const int par = l & 1;
    const unsigned long long* cur = par ? p.fr[1] : p.fr[0];
    unsigned long long* nxt = par ? p.fr[0] : p.fr[1];
    unsigned long long my_or = 0;
    // light vertices: one thread each.  The whole warp walks the range of
    // caller ids V0 together, so that the level and parent stores below (rows
    // of the caller's ids) coalesce; on a renumbered graph the lane pulls for
    // the internal vertex v = inv[V0].
    const long long n_round = (p.n + nthreads - 1) / nthreads * nthreads;
    for (long long V0 = tid; V0 < n_round; V0 += nthreads) {
      const long long v = (p.inv && V0 < p.n) ? __ldg(p.inv + V0) : V0;
      unsigned long long nw = 0;
      int b = 0;
      const bool mine = v < p.n && __ldg(rp + v + 1) - __ldg(rp + v) <= kMsHeavy;
      if (mine) {
        b = __ldg(rp + v);
        const int e = __ldg(rp + v + 1);
        const unsigned long long s = p.seen[v];
        const unsigned long long need = active & ~s;
        if (need) {
          unsigned long long acc = 0;
          for (int j = b; j < e && (acc & need) != need; j += kMsUnroll) {
            my_edges += min(kMsUnroll, e - j);
            int uu[kMsUnroll];
            unsigned long long ff[kMsUnroll];
#pragma unroll
            for (int t = 0; t < kMsUnroll; ++t) uu[t] = j + t < e ? __ldg(ci + j + t) : -1;
#pragma unroll
            for (int t = 0; t < kMsUnroll; ++t) ff[t] = uu[t] >= 0 ? ld_cg64(cur + uu[t]) : 0ull;
#pragma unroll
            for (int t = 0; t < kMsUnroll; ++t) {
              if (p.parents_out) {
                // the first neighbour carrying a new bit is its parent: note
                // its row offset, the store waits for the warp's bit loop
                unsigned long long c = ff[t] & ~s & ~acc;
                while (c) {
                  const int i = __ffsll((long long)c) - 1;
                  c &= c - 1;
                  s_off[i * kWarp + lane] = (uint8_t)(j + t - b);
                }
              }
              acc |= ff[t];
            }
          }
          nw = acc & ~s;
          if (nw) p.seen[v] = s | nw;
        }
        nxt[v] = nw;
        my_or |= nw;
      }
      // levels and parents of the new (source, vertex) pairs: one store per
      // source bit, shared by the lanes (consecutive vertices) that found
      // that source, so the source-major rows are written in runs
      unsigned long long wn = warp_or64(nw);
      if (wn) {
        const int V = (int)V0;
        while (wn) {
          const int i = __ffsll((long long)wn) - 1;
          wn &= wn - 1;
          if ((nw >> i) & 1ull) {
            p.levels_out[(long long)i * p.n + V] = l + 1;
            if (p.parents_out)
              p.parents_out[(long long)i * p.n + V] = out_id(p, __ldg(ci + b + s_off[i * kWarp + lane]));
          }
        }
      }
    }
    // heavy vertices: one warp each, neighbours 32 at a time in order
    for (int h = gw; h < p.n_heavy; h += nwarps) {
      const int v = __ldg(p.heavy + h);
      const int b = __ldg(rp + v), e = __ldg(rp + v + 1);
      const unsigned long long s = p.seen[v];
      const unsigned long long need = active & ~s;
      unsigned long long nw = 0;
      if (need) {
        const int V = out_id(p, v);
        unsigned long long acc = 0;
        for (int base = b; base < e && (acc & need) != need; base += kWarp) {  // acc is warp-uniform
          if (lane == 0) my_edges += min(kWarp, e - base);
          const int j = base + lane;
          int u = 0;
          unsigned long long f = 0;
          if (j < e) {
            u = __ldg(ci + j);
            f = ld_cg64(cur + u);
          }
          if (p.parents_out) {
            const unsigned long long c = f & ~s & ~(acc | warp_excl_or64(f, lane));
            if (c) write_bits(p, c, V, out_id(p, u), p.parents_out);
          }
          acc |= warp_or64(f);
        }
        nw = acc & ~s;
        if (nw) {
          if (lane == 0) p.seen[v] = s | nw;
          if ((nw >> lane) & 1ull) p.levels_out[(long long)lane * p.n + V] = l + 1;
          if ((nw >> (lane + 32)) & 1ull) p.levels_out[(long long)(lane + 32) * p.n + V] = l + 1;
        }
      }
      if (lane == 0) nxt[v] = nw;
      my_or |= nw;
    }
    // huge vertices: one CTA each; every warp pulls a slice of the
    // neighbours (a source found in several slices may get its parent written
    // more than once: every such parent is valid), the CTA ORs the slices
    for (int h = blockIdx.x; h < p.n_huge; h += gridDim.x) {
      const int v = __ldg(p.huge + h);
      const int b = __ldg(rp + v), e = __ldg(rp + v + 1);
      const unsigned long long s = p.seen[v];
      const unsigned long long need = active & ~s;
      unsigned long long acc = 0;
      if (need) {
        const int V = out_id(p, v);
        for (int base = b + wib * kWarp; base < e && (acc & need) != need; base += kWarpsPerCta * kWarp) {
          if (lane == 0) my_edges += min(kWarp, e - base);
          const int j = base + lane;
          int u = 0;
          unsigned long long f = 0;
          if (j < e) {
            u = __ldg(ci + j);
            f = ld_cg64(cur + u);
          }
          if (p.parents_out) {
            const unsigned long long c = f & ~s & ~(acc | warp_excl_or64(f, lane));
            if (c) write_bits(p, c, V, out_id(p, u), p.parents_out);
          }
          acc |= warp_or64(f);
        }
      }
      if (lane == 0) s_or[wib] = acc;
      __syncthreads();
      unsigned long long all = 0;
      for (int w = 0; w < kWarpsPerCta; ++w) all |= s_or[w];
      const unsigned long long nw = all & ~s;
      if (threadIdx.x == 0) {
        if (nw) p.seen[v] = s | nw;
        nxt[v] = nw;
      }
      if (nw && threadIdx.x < 64 && ((nw >> threadIdx.x) & 1ull))
        p.levels_out[(long long)threadIdx.x * p.n + out_id(p, v)] = l + 1;
      if (threadIdx.x == 0) my_or |= nw;
      __syncthreads();
    }
    // which sources found new vertices at this level, over the whole grid
    my_or = warp_or64(my_or);
    if (lane == 0) s_or[wib] = my_or;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long o = 0;
      for (int w = 0; w < kWarpsPerCta; ++w) o |= s_or[w];
      p.block_or[(long long)par * gridDim.x + blockIdx.x] = o;
    }
    if (!grid_sync(p, ++bar)) break;
    if (threadIdx.x == 0) {
      unsigned long long o = 0;
      for (int b2 = 0; b2 < (int)gridDim.x; ++b2) o |= ld_cg64(p.block_or + (long long)par * gridDim.x + b2);
      s_any = o;
      if (blockIdx.x == 0 && l < p.lvl_cap) p.level_bits[l] = o;
    }
    __syncthreads();
    const unsigned long long any = s_any;
    __syncthreads();
    if (any == 0) {
      finished = true;
      break;
    }
    active = any;  // the sources whose frontier the next level pulls
    ++l;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) p.st->num_levels = l + 1;
  if (finished && p.write_missing) {
    // every (source, vertex) pair the sources never reached gets -1, so each
    // output entry is written exactly once (no clearing pass beforehand).
    // seen[] is final: the last grid barrier orders every CTA's writes.  A
    // warp takes 32 consecutive caller ids; per source missing anywhere in
    // the warp, one store per array for the lanes that miss it.
    for (long long V0 = tid - lane; V0 < p.n; V0 += nthreads) {
      const long long V = V0 + lane;
      const long long v = V < p.n ? (p.inv ? __ldg(p.inv + V) : V) : 0;
      const unsigned long long miss = V < p.n ? full & ~ld_cg64(p.seen + v) : 0ull;
      unsigned long long wm = warp_or64(miss);
      while (wm) {
        const int i = __ffsll((long long)wm) - 1;
        wm &= wm - 1;
        if ((miss >> i) & 1ull) {
          p.levels_out[(long long)i * p.n + V] = -1;
          if (p.parents_out) p.parents_out[(long long)i * p.n + V] = -1;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) my_edges += __shfl_xor_sync(kFull, my_edges, o);
  if (lane == 0) s_edges[wib] = my_edges;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kWarpsPerCta; ++w) t += s_edges[w];
    p.block_edges[blockIdx.x] = t;
  }
}

// seen = frontier = 0 everywhere
__global__ void __launch_bounds__(kThreads) k_msbfs_clear(MsParams p) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
    p.seen[v] = 0ull;
    p.fr[0][v] = 0ull;
  }
}

// sources: grouped by vertex on the host (vs[j], masks[j] distinct vertices);
// src_int[i] / src_out[i] = internal and caller id of source i
__global__ void k_msbfs_sources(MsParams p, const int32_t* vs, const unsigned long long* masks, int groups,
                                const int32_t* src_int, const int32_t* src_out) {
  const int t = threadIdx.x;
  if (t < groups) {
    p.seen[vs[t]] = masks[t];
    p.fr[0][vs[t]] = masks[t];
  }
  if (t < p.k) {
    p.levels_out[(long long)t * p.n + src_out[t]] = 0;
    if (p.parents_out) p.parents_out[(long long)t * p.n + src_out[t]] = src_out[t];
  }
  if (t == 0) {
    p.st->err = 0;
    p.st->err_where = 0;
    p.st->bar_release = 0;
    p.st->num_levels = 0;
  }
}

// per source: reached vertices and the degree sum over them, partial per CTA
// (bit i of seen[v] counts for source i); out[b][i] and out[b][64 + i]
__global__ void __launch_bounds__(kThreads) k_msbfs_counts(MsParams p, long long* out) {
  __shared__ long long s_cnt[kWarpsPerCta][64];
  __shared__ long long s_deg[kWarpsPerCta][64];
  const int lane = threadIdx.x & (kWarp - 1);
  const int wib = threadIdx.x >> 5;
  long long cnt_lo = 0, cnt_hi = 0, deg_lo = 0, deg_hi = 0;  // bits lane and lane + 32
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x + wib * kWarp; base < p.n; base += stride) {
    const long long v = base + lane;
    unsigned long long s = 0;
    int d = 0;
    if (v < p.n) {
      s = p.seen[v];
      d = __ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v);
    }
    for (int i = 0; i < p.k; ++i) {
      const bool bit = (s >> i) & 1ull;
      const int c = __popc(__ballot_sync(kFull, bit));
      const int dd = __reduce_add_sync(kFull, bit ? d : 0);
      if (i < 32) {
        if (lane == i) { cnt_lo += c; deg_lo += dd; }
      } else {
        if (lane == i - 32) { cnt_hi += c; deg_hi += dd; }
      }
    }
  }
  s_cnt[wib][lane] = cnt_lo;
  s_cnt[wib][lane + 32] = cnt_hi;
  s_deg[wib][lane] = deg_lo;
  s_deg[wib][lane + 32] = deg_hi;
  __syncthreads();
  if (threadIdx.x < 64) {
    long long c = 0, dd = 0;
    for (int w = 0; w < kWarpsPerCta; ++w) {
      c += s_cnt[w][threadIdx.x];
      dd += s_deg[w][threadIdx.x];
    }
    out[(long long)blockIdx.x * 128 + threadIdx.x] = c;
    out[(long long)blockIdx.x * 128 + 64 + threadIdx.x] = dd;
  }
}

}  // namespace s3bfs
