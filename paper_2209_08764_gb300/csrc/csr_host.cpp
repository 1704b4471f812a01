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
