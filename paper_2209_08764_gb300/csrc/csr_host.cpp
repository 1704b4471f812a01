// Host-side CSR preparation for bfs_create_csr: the simple-graph check behind
// BFS_VALIDATE and the row clean-up behind BFS_DEDUP.
//
// The dedup step of the level loop keeps a candidate (v, u) when parent[v]
// still equals u; that identifies one survivor per newly reached vertex only
// if no row lists the same neighbour twice (the owner id of Fig. 1 lines
// 19-23 is taken to be the parent vertex), hence these checks.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <new>
#include <vector>

// Returns 0 if no row of the CSR repeats a neighbour, else 1 and a message.
int s3bfs_host_check_duplicates(int32_t n, const int32_t* rp, const int32_t* ci, char* msg, size_t len) {
  std::vector<int32_t> row;
  for (int32_t u = 0; u < n; ++u) {
    const int32_t b = rp[u], e = rp[u + 1];
    bool sorted = true;
    for (int32_t k = b + 1; k < e; ++k)
      if (ci[k] <= ci[k - 1]) {
        sorted = false;
        break;
      }
    if (sorted) continue;  // strictly increasing: no repeats
    row.assign(ci + b, ci + e);
    std::sort(row.begin(), row.end());
    for (size_t k = 1; k < row.size(); ++k)
      if (row[k] == row[k - 1]) {
        snprintf(msg, len, "row %d lists neighbour %d more than once", u, row[k]);
        return 1;
      }
  }
  return 0;
}

// Rewrites every row sorted ascending without repeated neighbours or
// self-loops.  Returns 0, or -1 if host memory ran out.
int s3bfs_host_dedup(int32_t n, const int32_t* rp, const int32_t* ci, std::vector<int32_t>* rp_out,
                     std::vector<int32_t>* ci_out) {
  try {
    rp_out->assign((size_t)n + 1, 0);
    ci_out->clear();
    ci_out->reserve((size_t)rp[n]);
    std::vector<int32_t> row;
    for (int32_t u = 0; u < n; ++u) {
      row.assign(ci + rp[u], ci + rp[u + 1]);
      std::sort(row.begin(), row.end());
      int32_t last = -1;
      for (int32_t v : row) {
        if (v == u || v == last) continue;
        ci_out->push_back(v);
        last = v;
      }
      (*rp_out)[(size_t)u + 1] = (int32_t)ci_out->size();
    }
    if (ci_out->empty()) ci_out->push_back(0);  // keep data() non-null; nnz comes from rp_out[n]
  } catch (const std::bad_alloc&) {
    return -1;
  }
  return 0;
}

// Share of all edge endpoints (sum of degrees) held by the `top` vertices of
// highest degree.
double s3bfs_host_top_degree_share(int32_t n, const int32_t* rp, int32_t top) {
  if (n <= 0 || rp[n] <= 0) return 0.0;
  if (top >= n) return 1.0;
  int32_t maxd = 0;
  for (int32_t v = 0; v < n; ++v) maxd = std::max(maxd, rp[v + 1] - rp[v]);
  std::vector<int64_t> cnt((size_t)maxd + 1, 0);
  for (int32_t v = 0; v < n; ++v) cnt[(size_t)(rp[v + 1] - rp[v])]++;
  int64_t left = top, sum = 0;
  for (int32_t d = maxd; d >= 0 && left > 0; --d) {
    const int64_t take = std::min<int64_t>(left, cnt[(size_t)d]);
    sum += take * d;
    left -= take;
  }
  return (double)sum / (double)rp[n];
}

// Degree-descending renumbering (ties by id): perm[i] is the caller's id of
// internal vertex i, inv[v] the internal id of v.  The renumbered CSR lists
// internal rows in order, with every neighbour translated through inv; with
// sort_rows every row is sorted (highest-degree neighbours first, which a
// bottom-up level tries first).  Returns 0, or -1 if host memory ran out.
int s3bfs_host_relabel(int32_t n, const int32_t* rp, const int32_t* ci, bool sort_rows, std::vector<int32_t>* perm,
                       std::vector<int32_t>* inv, std::vector<int32_t>* rp_out, std::vector<int32_t>* ci_out) {
  try {
    int32_t maxd = 0;
    for (int32_t v = 0; v < n; ++v) maxd = std::max(maxd, rp[v + 1] - rp[v]);
    // counting sort by degree, descending; stable in the id
    std::vector<int64_t> start((size_t)maxd + 2, 0);
    for (int32_t v = 0; v < n; ++v) start[(size_t)(maxd - (rp[v + 1] - rp[v])) + 1]++;
    for (size_t d = 1; d < start.size(); ++d) start[d] += start[d - 1];
    perm->assign((size_t)n, 0);
    inv->assign((size_t)n, 0);
    for (int32_t v = 0; v < n; ++v) {
      const int64_t i = start[(size_t)(maxd - (rp[v + 1] - rp[v]))]++;
      (*perm)[(size_t)i] = v;
      (*inv)[(size_t)v] = (int32_t)i;
    }
    rp_out->assign((size_t)n + 1, 0);
    ci_out->assign((size_t)std::max(rp[n], 1), 0);
    int64_t w = 0;
    for (int32_t i = 0; i < n; ++i) {
      const int32_t v = (*perm)[(size_t)i];
      const int64_t w0 = w;
      for (int32_t e = rp[v]; e < rp[v + 1]; ++e) (*ci_out)[(size_t)w++] = (*inv)[(size_t)ci[e]];
      if (sort_rows) std::sort(ci_out->begin() + w0, ci_out->begin() + w);
      (*rp_out)[(size_t)i + 1] = (int32_t)w;
    }
  } catch (const std::bad_alloc&) {
    return -1;
  }
  return 0;
}

// True if every edge (u, v) has its reverse (v, u).  Rows are sorted in a
// copy where needed, then every reverse edge is found by binary search.
int s3bfs_host_is_symmetric(int32_t n, const int32_t* rp, const int32_t* ci) {
  std::vector<int32_t> sorted(ci, ci + rp[n]);
  for (int32_t u = 0; u < n; ++u) std::sort(sorted.begin() + rp[u], sorted.begin() + rp[u + 1]);
  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
      const int32_t v = sorted[(size_t)e];
      if (!std::binary_search(sorted.begin() + rp[v], sorted.begin() + rp[v + 1], u)) return 0;
    }
  return 1;
}
