/*
 * CPU oracle for breadth-first search levels -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file; the CUDA library never links or calls it, and it shares no code,
 * header or helper with the CUDA path.
 *
 * What it computes: the array the paper's Parallel-BFS(s, P) returns (Fig. 1,
 * header: d[0:n-1], the distance from s to every vertex; Introduction: a
 * level-synchronous BFS explores the first-level neighbours of s, then the
 * second level, and so on).  That array has a plain definition -- the hop
 * distance from s, or "infinity" when v is unreachable -- so the oracle is
 * that definition written out as the textbook sequential FIFO-queue BFS:
 *
 *   d[*] = -1 (stands for infinity), parent[*] = -1, d[s] = 0, parent[s] = s,
 *   push s; while the queue is non-empty: pop u; for each out-neighbour v of u
 *   in CSR order: if d[v] == -1 then d[v] = d[u] + 1, parent[v] = u, push v.
 *
 * The parent array is not in the paper (which returns d only); it is the BFS
 * tree recorded alongside, used only as one valid tree among many.
 */
#include <stdint.h>
#include <stdlib.h>

/* Returns the number of reached vertices (including s), or -1 on bad
 * arguments.  `queue` is caller scratch of n int32 entries; `parent` may be
 * NULL. */
int64_t oracle_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t s,
                   int32_t *level, int32_t *parent, int32_t *queue) {
  if (n <= 0 || s < 0 || s >= n || !row_ptr || !level || !queue) return -1;
  for (int32_t v = 0; v < n; ++v) level[v] = -1;
  if (parent)
    for (int32_t v = 0; v < n; ++v) parent[v] = -1;
  int64_t head = 0, tail = 0;
  level[s] = 0;
  if (parent) parent[s] = s;
  queue[tail++] = s;
  while (head < tail) {
    const int32_t u = queue[head++];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      const int32_t v = col_idx[e];
      if (level[v] == -1) {
        level[v] = level[u] + 1;
        if (parent) parent[v] = u;
        queue[tail++] = v;
      }
    }
  }
  return tail;
}
