// Reverse Cuthill-McKee node order (host code; the relabelling option
// reorder = 2 of wl_build, and wl_rcm_order in the C ABI).
//
// Cuthill-McKee numbers the nodes of each connected component in
// breadth-first order from a pseudo-peripheral start node, appending the
// unnumbered neighbours of every node by increasing degree (ties by node
// id); reversing the whole numbering (George) keeps the bandwidth and
// shrinks the profile. Nearby labels then mean nearby nodes, so the rows a
// CTA gathers share neighbours in L2. The start node of a component is found
// by the usual level-structure search: from the component's lowest-degree
// node, repeatedly restart from the lowest-degree node of the last BFS level
// while the eccentricity grows (at most kPeripheralRounds restarts).
// Components are taken in order of their lowest-degree node (ties by id).
// Deterministic; O(nnz log dmax) time, O(n) extra memory besides the
// neighbour buffer.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "wl.h"
#include "wl_host.h"

namespace wl {

namespace {

constexpr int kPeripheralRounds = 8;

// BFS levels from r (over r's connected component); returns the eccentricity
// of r and leaves the nodes of the last level in `last`
int bfs_levels(const int32_t* rp, const int32_t* col, int32_t r, std::vector<int32_t>& level,
               std::vector<int32_t>& queue, std::vector<int32_t>& touched, std::vector<int32_t>& last) {
  for (int32_t v : touched) level[v] = -1;
  touched.clear();
  queue.clear();
  queue.push_back(r);
  level[r] = 0;
  touched.push_back(r);
  size_t head = 0;
  int ecc = 0;
  while (head < queue.size()) {
    const int32_t u = queue[head++];
    for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
      const int32_t v = col[e];
      if (level[v] < 0) {
        level[v] = level[u] + 1;
        ecc = std::max(ecc, level[v]);
        queue.push_back(v);
        touched.push_back(v);
      }
    }
  }
  last.clear();
  for (int32_t v : queue)
    if (level[v] == ecc) last.push_back(v);
  return ecc;
}

}  // namespace

int rcm_order(const int32_t* rp, const int32_t* col, int64_t n, int32_t* perm) {
  if (n < 0 || (n > 0 && (!rp || !perm)) || (n > 0 && rp[n] > 0 && !col)) return WL_ERR_INVALID_ARG;
  if (n == 0) return WL_OK;
  auto deg = [&](int32_t v) { return rp[v + 1] - rp[v]; };
  // candidate starts: nodes by increasing degree, ties by id
  std::vector<int32_t> byd((size_t)n);
  std::iota(byd.begin(), byd.end(), 0);
  std::stable_sort(byd.begin(), byd.end(), [&](int32_t a, int32_t b) { return deg(a) < deg(b); });
  std::vector<char> numbered((size_t)n, 0);
  std::vector<int32_t> level((size_t)n, -1), queue, touched, last, nbr;
  queue.reserve((size_t)n);
  std::vector<int32_t> order;
  order.reserve((size_t)n);
  for (int32_t s : byd) {
    if (numbered[s]) continue;
    // pseudo-peripheral start of s's component
    int32_t r = s;
    int ecc = bfs_levels(rp, col, r, level, queue, touched, last);
    for (int round = 0; round < kPeripheralRounds; ++round) {
      int32_t x = last[0];
      for (int32_t v : last)
        if (deg(v) < deg(x) || (deg(v) == deg(x) && v < x)) x = v;
      const int e2 = bfs_levels(rp, col, x, level, queue, touched, last);
      if (e2 <= ecc) break;
      r = x;
      ecc = e2;
    }
    // Cuthill-McKee from r
    const size_t first = order.size();
    order.push_back(r);
    numbered[r] = 1;
    for (size_t head = first; head < order.size(); ++head) {
      const int32_t u = order[head];
      nbr.clear();
      for (int32_t e = rp[u]; e < rp[u + 1]; ++e)
        if (!numbered[col[e]]) {
          numbered[col[e]] = 1;
          nbr.push_back(col[e]);
        }
      std::sort(nbr.begin(), nbr.end(),
                [&](int32_t a, int32_t b) { return deg(a) < deg(b) || (deg(a) == deg(b) && a < b); });
      order.insert(order.end(), nbr.begin(), nbr.end());
    }
  }
  // reversed numbering: perm[new] = old
  for (int64_t i = 0; i < n; ++i) perm[i] = order[(size_t)(n - 1 - i)];
  return WL_OK;
}

}  // namespace wl

extern "C" int wl_rcm_order(const int32_t* row_ptr, const int32_t* col_idx, int64_t n, int32_t* perm) {
  return wl::rcm_order(row_ptr, col_idx, n, perm);
}
