// Band-reducing ordering of the free-unknown graph for the banded direct
// solver: reverse Cuthill-McKee (Cuthill & McKee 1969; reversal by George
// 1971), a breadth-first numbering with neighbours taken in increasing degree,
// then reversed.  Two start sets are tried and the narrower band is kept:
//  * a pseudo-peripheral node (found by repeated breadth-first searches,
//    Gibbs-Poole-Stockmeyer style), the textbook choice;
//  * when the free nodes next to the Dirichlet boundary form two or more
//    connected pieces (an annulus: the inner and the outer circle), a
//    shortest path between two of them.  Numbering outwards from such a path
//    cuts a ring-shaped domain open along it: every level is then two thin
//    strips parallel to the path instead of the slanted fronts that grow from
//    one node, which on the machine-like annuli narrows the band by a third
//    (e.g. 204 -> 137 on the 20k-node annulus).
// Host code; runs once per mesh.
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

// Cuthill-McKee numbering from the start set `start` (level 0, in the given
// order) over the nodes not yet done, appended to `order`.
void cm_levels(const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
               const std::vector<int32_t>& deg, const std::vector<int32_t>& start,
               std::vector<char>& done, std::vector<int32_t>& order) {
  std::queue<int32_t> q;
  for (int v : start)
    if (!done[v]) {
      done[v] = 1;
      q.push(v);
    }
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

// Remaining components from pseudo-peripheral nodes (textbook RCM start).
void cm_rest(int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
             const std::vector<int32_t>& deg, std::vector<char>& done,
             std::vector<int32_t>& order) {
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
    cm_levels(rp, ci, deg, {start}, done, order);
  }
}

// Reversal of a Cuthill-McKee order and its bandwidth.
int32_t reverse_and_width(int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                          const std::vector<int32_t>& order, std::vector<int32_t>& perm) {
  perm.assign(order.rbegin(), order.rend());
  std::vector<int32_t> iperm(n);
  for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
  int32_t bw = 0;
  for (int v = 0; v < n; ++v)
    for (int k = rp[v]; k < rp[v + 1]; ++k) bw = std::max(bw, std::abs(iperm[v] - iperm[ci[k]]));
  return bw;
}

// A shortest path between two connected pieces of the boundary-adjacent
// nodes (empty when there are fewer than two pieces).
std::vector<int32_t> boundary_path(int n, const std::vector<int32_t>& rp,
                                   const std::vector<int32_t>& ci,
                                   const std::vector<char>& boundary) {
  if ((int)boundary.size() != n) return {};
  std::vector<int32_t> piece(n, -1);
  int n_pieces = 0;
  for (int v = 0; v < n; ++v) {
    if (!boundary[v] || piece[v] >= 0) continue;
    std::vector<int32_t> stack{v};
    piece[v] = n_pieces;
    while (!stack.empty()) {
      const int x = stack.back();
      stack.pop_back();
      for (int k = rp[x]; k < rp[x + 1]; ++k)
        if (boundary[ci[k]] && piece[ci[k]] < 0) {
          piece[ci[k]] = n_pieces;
          stack.push_back(ci[k]);
        }
    }
    ++n_pieces;
  }
  if (n_pieces < 2) return {};
  // breadth-first search from all of piece 0 to the nearest node of another piece
  std::vector<int32_t> parent(n, -2);
  std::queue<int32_t> q;
  for (int v = 0; v < n; ++v)
    if (piece[v] == 0) {
      parent[v] = -1;
      q.push(v);
    }
  int hit = -1;
  while (!q.empty() && hit < 0) {
    const int x = q.front();
    q.pop();
    for (int k = rp[x]; k < rp[x + 1]; ++k) {
      const int u = ci[k];
      if (parent[u] != -2) continue;
      parent[u] = x;
      if (piece[u] > 0) {
        hit = u;
        break;
      }
      q.push(u);
    }
  }
  std::vector<int32_t> path;
  for (int v = hit; v >= 0; v = parent[v]) path.push_back(v);
  return path;
}

}  // namespace

void rcm_order(int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
               const std::vector<char>& boundary, std::vector<int32_t>& perm,
               int32_t& bandwidth) {
  std::vector<int32_t> deg(n);
  for (int v = 0; v < n; ++v) deg[v] = rp[v + 1] - rp[v];
  // textbook start: a pseudo-peripheral node per component
  std::vector<char> done(n, 0);
  std::vector<int32_t> order;
  order.reserve(n);
  cm_rest(n, rp, ci, deg, done, order);
  bandwidth = reverse_and_width(n, rp, ci, order, perm);
  // start set: a shortest path between two pieces of the boundary
  const std::vector<int32_t> path = boundary_path(n, rp, ci, boundary);
  if (path.empty()) return;
  std::fill(done.begin(), done.end(), 0);
  order.clear();
  cm_levels(rp, ci, deg, path, done, order);
  cm_rest(n, rp, ci, deg, done, order);
  std::vector<int32_t> perm2;
  const int32_t bw2 = reverse_and_width(n, rp, ci, order, perm2);
  if (bw2 < bandwidth) {
    bandwidth = bw2;
    perm.swap(perm2);
  }
}

}  // namespace mqs
