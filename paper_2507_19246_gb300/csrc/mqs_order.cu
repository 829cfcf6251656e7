// Reverse Cuthill-McKee ordering (Cuthill & McKee 1969; reversal by George
// 1971) of the free-unknown graph, used by the banded direct solver: a
// breadth-first numbering from a pseudo-peripheral node (found by repeated
// breadth-first searches, Gibbs-Poole-Stockmeyer style), neighbours taken in
// increasing degree, then reversed.  Host code; runs once per mesh.
#include "mqs_internal.cuh"

#include <algorithm>
#include <queue>

namespace mqs {
namespace {

// Breadth-first levels from `start` over unvisited nodes; returns the last level.
int bfs_depth(int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci, int start,
              std::vector<int32_t>& level, std::vector<int32_t>& last) {
  std::fill(level.begin(), level.end(), -1);
  std::vector<int32_t> cur{start}, nxt;
  level[start] = 0;
  int depth = 0;
  last = cur;
  while (!cur.empty()) {
    nxt.clear();
    for (int v : cur)
      for (int k = rp[v]; k < rp[v + 1]; ++k) {
        const int u = ci[k];
        if (level[u] < 0) {
          level[u] = depth + 1;
          nxt.push_back(u);
        }
      }
    if (nxt.empty()) break;
    last = nxt;
    cur.swap(nxt);
    ++depth;
  }
  return depth;
}

}  // namespace

void rcm_order(int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
               std::vector<int32_t>& perm, int32_t& bandwidth) {
  std::vector<int32_t> deg(n);
  for (int v = 0; v < n; ++v) deg[v] = rp[v + 1] - rp[v];
  std::vector<char> done(n, 0);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<int32_t> level(n), last;
  for (int seed = 0; seed < n; ++seed) {
    if (done[seed]) continue;
    // pseudo-peripheral start node within this component
    int start = seed;
    for (int v = seed; v < n; ++v)
      if (!done[v] && deg[v] < deg[start]) start = v;
    int ecc = bfs_depth(n, rp, ci, start, level, last);
    for (int it = 0; it < 8; ++it) {
      int cand = last[0];
      for (int v : last)
        if (deg[v] < deg[cand]) cand = v;
      const int e2 = bfs_depth(n, rp, ci, cand, level, last);
      if (e2 <= ecc) break;
      ecc = e2;
      start = cand;
    }
    // Cuthill-McKee numbering
    std::queue<int32_t> q;
    q.push(start);
    done[start] = 1;
    std::vector<int32_t> nb;
    while (!q.empty()) {
      const int v = q.front();
      q.pop();
      order.push_back(v);
      nb.clear();
      for (int k = rp[v]; k < rp[v + 1]; ++k)
        if (!done[ci[k]]) nb.push_back(ci[k]);
      std::sort(nb.begin(), nb.end(), [&](int a, int b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
      for (int u : nb) {
        done[u] = 1;
        q.push(u);
      }
    }
  }
  perm.assign(order.rbegin(), order.rend());
  std::vector<int32_t> iperm(n);
  for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
  bandwidth = 0;
  for (int v = 0; v < n; ++v)
    for (int k = rp[v]; k < rp[v + 1]; ++k)
      bandwidth = std::max(bandwidth, std::abs(iperm[v] - iperm[ci[k]]));
}

}  // namespace mqs
