// Approximate minimum degree ordering (Amestoy, Davis and Duff, SIAM J.
// Matrix Anal. Appl. 17(4), 1996), written for the KKT matrices of this
// solver.  It runs once at setup on the host.
//
// Quotient-graph formulation: eliminated pivots become "elements"; a variable
// i keeps a list E[i] of adjacent elements and a list A[i] of adjacent
// variables that are not yet covered by an element.  At each step the
// variable of least approximate external degree is eliminated; its element
// L_p = A_p u (union of L_e, e in E_p) \ {p} absorbs the elements in E_p.
// Degrees of the variables in L_p are bounded by
//     d_i <= min(nleft - |i|, d_i_old + |L_p \ i|,
//                |A_i \ i| + |L_p \ i| + sum_{e in E_i \ p} |L_e \ L_p|),
// where |L_e \ L_p| is obtained for all e at once by scanning L_p.
// Variables with identical adjacency are merged into supervariables
// (hashing), elements with L_e inside L_p are absorbed (aggressive
// absorption), and nodes of degree > max(16, 10 sqrt(N)) are ordered last.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace clr {

namespace {

enum { VAR = 0, ELEM = 1, MERGED = 2, DEAD = 3, DENSE = 4 };

// splitmix64 finaliser: spreads an index over 64 bits for the order-free list hash
inline uint64_t mix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

struct DegreeLists {
  std::vector<int64_t> head, next, prev;
  int64_t mindeg = 0;
  explicit DegreeLists(int64_t N) : head(N + 1, -1), next(N, -1), prev(N, -1) {}
  void insert(int64_t i, int64_t d) {
    next[i] = head[d];
    prev[i] = -1;
    if (head[d] >= 0) prev[head[d]] = i;
    head[d] = i;
    if (d < mindeg) mindeg = d;
  }
  void remove(int64_t i, int64_t d) {
    if (prev[i] >= 0) next[prev[i]] = next[i];
    else head[d] = next[i];
    if (next[i] >= 0) prev[next[i]] = prev[i];
    next[i] = prev[i] = -1;
  }
};

}  // namespace

void amd_order(int64_t N, const std::vector<int64_t>& ptr, const std::vector<int64_t>& idx,
               std::vector<int64_t>& perm, int64_t& n_dense) {
  perm.clear();
  perm.reserve(N);
  n_dense = 0;
  if (N == 0) return;
  std::vector<std::vector<int64_t>> A(N), E(N), Le(N), members(N);
  std::vector<int64_t> nv(N, 1), deg(N, 0), status(N, VAR);
  for (int64_t i = 0; i < N; ++i) {
    for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p)
      if (idx[p] != i) A[i].push_back(idx[p]);
    deg[i] = (int64_t)A[i].size();
    members[i].push_back(i);
  }
  const double dense_thresh = std::max(16.0, 10.0 * std::sqrt((double)N));
  std::vector<int64_t> dense_nodes;
  for (int64_t i = 0; i < N; ++i)
    if ((double)deg[i] > dense_thresh && N > 16) {
      status[i] = DENSE;
      dense_nodes.push_back(i);
    }
  n_dense = (int64_t)dense_nodes.size();
  // drop dense nodes from adjacency, recompute degrees
  for (int64_t i = 0; i < N; ++i) {
    if (status[i] == DENSE) continue;
    std::vector<int64_t>& a = A[i];
    a.erase(std::remove_if(a.begin(), a.end(), [&](int64_t v) { return status[v] == DENSE; }), a.end());
    deg[i] = (int64_t)a.size();
  }
  DegreeLists dl(N);
  dl.mindeg = N;
  for (int64_t i = 0; i < N; ++i)
    if (status[i] == VAR) dl.insert(i, deg[i]);

  std::vector<int64_t> mark(N, -1), wtag(N, -1), wval(N, 0), ew(N, 0);
  int64_t tag = 0;
  int64_t nleft = N - n_dense;  // weighted count of uneliminated variables
  std::vector<int64_t> Lp, group;
  std::vector<uint64_t> hv(N, 0);
  std::vector<std::pair<uint64_t, int64_t>> hashed;
  while (nleft > 0) {
    // ---- select pivot of minimum approximate degree ----
    while (dl.mindeg <= N && dl.head[dl.mindeg] < 0) ++dl.mindeg;
    const int64_t p = dl.head[dl.mindeg];
    dl.remove(p, deg[p]);
    ++tag;
    // ---- L_p = (A_p u union L_e) \ p; absorb E_p ----
    Lp.clear();
    mark[p] = tag;
    int64_t wLp = 0;
    for (int64_t e : E[p]) {
      if (status[e] != ELEM) continue;
      for (int64_t v : Le[e])
        if (status[v] == VAR && mark[v] != tag) {
          mark[v] = tag;
          Lp.push_back(v);
          wLp += nv[v];
        }
      status[e] = DEAD;
      std::vector<int64_t>().swap(Le[e]);
    }
    for (int64_t v : A[p])
      if (status[v] == VAR && mark[v] != tag) {
        mark[v] = tag;
        Lp.push_back(v);
        wLp += nv[v];
      }
    std::vector<int64_t>().swap(A[p]);
    std::vector<int64_t>().swap(E[p]);
    status[p] = ELEM;
    for (int64_t v : members[p]) perm.push_back(v);
    std::vector<int64_t>().swap(members[p]);
    nleft -= nv[p];
    Le[p] = Lp;
    ew[p] = wLp;

    // ---- |L_e \ L_p| for every element e adjacent to L_p ----
    for (int64_t i : Lp) {
      for (int64_t e : E[i]) {
        if (status[e] != ELEM || e == p) continue;
        if (wtag[e] != tag) {
          // |L_e| (weighted) is fixed for the life of e: a variable of L_e that is
          // eliminated absorbs e, and a merge moves weight between two members
          wtag[e] = tag;
          wval[e] = ew[e];
        }
        wval[e] -= nv[i];
      }
    }
    // ---- update each variable in L_p ----
    for (int64_t i : Lp) {
      dl.remove(i, deg[i]);
      std::vector<int64_t>& Ei = E[i];
      int64_t ext = 0;
      size_t o = 0;
      uint64_t h = 0;  // order-free hash of E[i] and A[i] for the supervariable test
      for (size_t t = 0; t < Ei.size(); ++t) {
        int64_t e = Ei[t];
        if (status[e] != ELEM || e == p) continue;
        if (wtag[e] == tag && wval[e] <= 0) {  // aggressive absorption: L_e inside L_p
          status[e] = DEAD;
          std::vector<int64_t>().swap(Le[e]);
          continue;
        }
        Ei[o++] = e;
        ext += (wtag[e] == tag) ? wval[e] : 0;
        h += mix64((uint64_t)e);
      }
      Ei.resize(o);
      Ei.push_back(p);
      h += mix64((uint64_t)p);
      std::vector<int64_t>& Ai = A[i];
      int64_t wA = 0;
      o = 0;
      for (size_t t = 0; t < Ai.size(); ++t) {
        int64_t v = Ai[t];
        if (status[v] != VAR || mark[v] == tag || v == i) continue;  // covered by element p
        Ai[o++] = v;
        wA += nv[v];
        h += mix64((uint64_t)v ^ 0x9e3779b97f4a7c15ull);
      }
      Ai.resize(o);
      hv[i] = h;
      const int64_t lp_i = wLp - nv[i];
      int64_t d = std::min(nleft - nv[i], deg[i] + lp_i);
      d = std::min(d, wA + lp_i + ext);
      deg[i] = std::max<int64_t>(d, 0);
    }
    // ---- supervariables: merge variables of L_p with identical adjacency ----
    if (Lp.size() > 1) {
      // candidates grouped by the hash taken in the update above (a group keeps the
      // order of L_p; equal lists always share a group, and only equal lists merge)
      hashed.clear();
      for (size_t t = 0; t < Lp.size(); ++t) {
        // E[i] is sorted but for the element p just appended, A[i] is sorted (compaction
        // keeps the order): one insertion instead of a sort
        std::vector<int64_t>& Ei = E[Lp[t]];
        if (!Ei.empty()) std::rotate(std::upper_bound(Ei.begin(), Ei.end() - 1, Ei.back()), Ei.end() - 1, Ei.end());
        hashed.emplace_back(hv[Lp[t]], (int64_t)t);
      }
      std::sort(hashed.begin(), hashed.end());
      for (size_t g0 = 0; g0 < hashed.size();) {
        size_t g1 = g0 + 1;
        while (g1 < hashed.size() && hashed[g1].first == hashed[g0].first) ++g1;
        group.clear();
        for (size_t t = g0; t < g1; ++t) group.push_back(Lp[hashed[t].second]);
        g0 = g1;
        const std::vector<int64_t>& g = group;
        for (size_t a = 0; a < g.size(); ++a) {
          int64_t i = g[a];
          if (status[i] != VAR) continue;
          for (size_t b2 = a + 1; b2 < g.size(); ++b2) {
            int64_t j = g[b2];
            if (status[j] != VAR) continue;
            // i and j are adjacent to each other only through elements (the A lists
            // exclude L_p, to which both belong), so their lists compare as they are
            if (E[i] == E[j] && A[i] == A[j]) {
              nv[i] += nv[j];
              deg[i] = std::max<int64_t>(deg[i] - nv[j], 0);
              nv[j] = 0;
              status[j] = MERGED;
              members[i].insert(members[i].end(), members[j].begin(), members[j].end());
              std::vector<int64_t>().swap(members[j]);
              std::vector<int64_t>().swap(A[j]);
              std::vector<int64_t>().swap(E[j]);
            }
          }
        }
      }
    }
    for (int64_t i : Lp)
      if (status[i] == VAR) {
        if (deg[i] > N) deg[i] = N;
        dl.insert(i, deg[i]);
      }
    // L_p keeps only principal variables
    std::vector<int64_t>& le = Le[p];
    le.erase(std::remove_if(le.begin(), le.end(), [&](int64_t v) { return status[v] != VAR; }), le.end());
  }
  for (int64_t v : dense_nodes) perm.push_back(v);
}

}  // namespace clr
