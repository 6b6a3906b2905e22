// Symbolic analysis of the KKT matrix, once at setup, on the host:
// fill-reducing order (AMD), elimination tree, postorder, column structures,
// fundamental supernodes, the supernodal tree and its level schedule, the
// layout of the frontal-matrix pool, and the index maps the numeric phase
// needs.  The numeric LDL^T is multifrontal: front J is a dense f_J x f_J
// block holding rows_J (own columns first); its first c_J columns become the
// panel of L, its trailing r_J x r_J block the update matrix that the parent
// front gathers ("extend-add") before its own elimination.
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <atomic>
#include <exception>
#include <mutex>
#include <queue>
#include <system_error>
#include <thread>

#include "internal.h"
#include "symbolic.h"

namespace clr {

namespace {
// Symmetric adjacency (no diagonal) of the matrix whose lower triangle is given as CSC.
void build_adjacency(int64_t N, const std::vector<int64_t>& colptr, const std::vector<int64_t>& rowidx,
                     std::vector<int64_t>& aptr, std::vector<int64_t>& aidx) {
  std::vector<int64_t> deg(N, 0);
  for (int64_t j = 0; j < N; ++j)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      int64_t i = rowidx[p];
      if (i == j) continue;
      deg[i]++;
      deg[j]++;
    }
  aptr.assign(N + 1, 0);
  for (int64_t i = 0; i < N; ++i) aptr[i + 1] = aptr[i] + deg[i];
  aidx.assign(aptr[N], 0);
  std::vector<int64_t> next(aptr.begin(), aptr.end() - 1);
  for (int64_t j = 0; j < N; ++j)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      int64_t i = rowidx[p];
      if (i == j) continue;
      aidx[next[i]++] = j;
      aidx[next[j]++] = i;
    }
}
}  // namespace

void kkt_amd_order(int64_t N, const std::vector<int64_t>& colptr, const std::vector<int64_t>& rowidx,
                   std::vector<int64_t>& order, int64_t& n_dense) {
  std::vector<int64_t> aptr, aidx;
  build_adjacency(N, colptr, rowidx, aptr, aidx);
  amd_order(N, aptr, aidx, order, n_dense);
}

namespace {
// Column counts of the factor of the symmetric pattern (aptr/aidx) eliminated in
// `order`, without forming the factor: elimination tree, postorder, then the
// row-subtree skeleton count of Gilbert, Ng and Peyton -- for every row i the
// leaves of its row subtree add +1 and the lowest common ancestor of two
// consecutive leaves -1, so that a subtree sum gives each column's count.
// Returns nnz(L) (diagonal included) and the flop count used by the symbolic.
void factor_counts(int64_t N, const std::vector<int64_t>& aptr, const std::vector<int64_t>& aidx,
                   const std::vector<int64_t>& order, int64_t* nnz, double* flops) {
  std::vector<int64_t> iorder(N);
  for (int64_t k = 0; k < N; ++k) iorder[order[k]] = k;
  std::vector<int64_t> parent(N, -1), anc(N, -1);
  for (int64_t k = 0; k < N; ++k) {
    const int64_t v = order[k];
    for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) {
      int64_t i = iorder[aidx[p]];
      if (i >= k) continue;
      while (i != -1 && i != k) {
        const int64_t nxt = anc[i];
        anc[i] = k;
        if (nxt == -1) parent[i] = k;
        i = nxt;
      }
    }
  }
  // postorder
  std::vector<int64_t> head(N, -1), nextc(N, -1), post;
  post.reserve(N);
  for (int64_t j = N - 1; j >= 0; --j)
    if (parent[j] >= 0) {
      nextc[j] = head[parent[j]];
      head[parent[j]] = j;
    }
  std::vector<int64_t> stack;
  for (int64_t r = 0; r < N; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      const int64_t top = stack.back();
      const int64_t c = head[top];
      if (c != -1) {
        head[top] = nextc[c];
        stack.push_back(c);
      } else {
        post.push_back(top);
        stack.pop_back();
      }
    }
  }
  // first[j]: smallest postorder index in the subtree of j; leaves have first == own index
  std::vector<int64_t> kpos(N), first(N, -1), delta(N, 0);
  for (int64_t k = 0; k < N; ++k) kpos[post[k]] = k;
  for (int64_t k = 0; k < N; ++k) {
    int64_t j = post[k];
    delta[j] = (first[j] == -1) ? 1 : 0;  // leaf of the elimination tree
    for (; j != -1 && first[j] == -1; j = parent[j]) first[j] = k;
  }
  std::vector<int64_t> maxfirst(N, -1), prevleaf(N, -1), setp(N);
  for (int64_t i = 0; i < N; ++i) setp[i] = i;
  auto find = [&](int64_t x) {
    int64_t r = x;
    while (setp[r] != r) r = setp[r];
    while (setp[x] != r) {
      const int64_t nx = setp[x];
      setp[x] = r;
      x = nx;
    }
    return r;
  };
  for (int64_t k = 0; k < N; ++k) {
    const int64_t j = post[k];
    if (parent[j] != -1) delta[parent[j]] -= 1;
    const int64_t v = order[j];
    for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) {
      const int64_t i = iorder[aidx[p]];  // entry (i, j) of the lower triangle when i > j
      if (i <= j) continue;
      if (first[j] <= maxfirst[i]) continue;  // j is not a leaf of row subtree i
      maxfirst[i] = first[j];
      const int64_t jprev = prevleaf[i];
      prevleaf[i] = j;
      delta[j] += 1;
      if (jprev != -1) delta[find(jprev)] -= 1;  // lca of consecutive leaves
    }
    if (parent[j] != -1) setp[j] = parent[j];
  }
  for (int64_t k = 0; k < N; ++k) {
    const int64_t j = post[k];
    if (parent[j] != -1) delta[parent[j]] += delta[j];
  }
  int64_t nz = 0;
  double fl = 0;
  for (int64_t j = 0; j < N; ++j) {
    nz += delta[j];
    const double below = (double)(delta[j] - 1);
    fl += below * (below + 1.0) + below;
  }
  (void)kpos;
  *nnz = nz;
  *flops = fl;
}
}  // namespace

void kkt_factor_counts(int64_t N, const std::vector<int64_t>& colptr, const std::vector<int64_t>& rowidx,
                       const std::vector<int64_t>& order, int64_t* nnz, double* flops) {
  std::vector<int64_t> aptr, aidx;
  build_adjacency(N, colptr, rowidx, aptr, aidx);
  factor_counts(N, aptr, aidx, order, nnz, flops);
}

// Fill-reducing order of one problem's KKT matrix.  Two candidates, the one
// whose factor needs fewer flops wins (ties: AMD):
//   0  AMD on the whole KKT pattern;
//   1  the constraint rows with a nonzero H block (nonnegative and cone rows)
//      first, in row order -- H is block diagonal, so they cause no fill among
//      themselves -- then x, the zero-cone rows and the auxiliary rows of the
//      expanded SOCs in the AMD order of their Schur-complement pattern (K
//      restricted to them, plus one clique per H block over the x columns its
//      rows touch; an expanded SOC's rows are 1 x 1 blocks whose cliques also
//      hold the cone's two auxiliary rows).
// AMD alone eliminates the low-degree x columns of a sparse random A first and
// fills the whole constraint block; candidate 1 leaves a dense x block instead.
int choose_kkt_order(const HostProblem& hp, std::vector<int64_t>& order, int64_t& n_dense, int* which) {
  const int64_t n = hp.n, m = hp.m, N = n + m;
  std::vector<int64_t> aptr, aidx;
  build_adjacency(N, hp.kcol_ptr, hp.krow, aptr, aidx);
  *which = 0;
  const int64_t mz = hp.cl.m_zero, ab = hp.cl.n_aux ? hp.cl.aux_begin : m, na = hp.cl.n_aux;
  if (ab - mz <= 0 || n == 0) {
    amd_order(N, aptr, aidx, order, n_dense);
    return CLR_OK;
  }
  // candidate 0 (AMD on the whole pattern and its flop count) on a second thread
  // while candidate 1 is built here, for patterns large enough to repay the thread;
  // the two only read the shared adjacency, so the result is the one a sequential
  // run gives
  int64_t nz0 = 0;
  double f0 = 0;
  std::exception_ptr err0;
  auto cand0 = [&] {
    try {
      amd_order(N, aptr, aidx, order, n_dense);
      factor_counts(N, aptr, aidx, order, &nz0, &f0);
    } catch (...) {
      err0 = std::current_exception();
    }
  };
  std::thread th;
  if ((int64_t)aidx.size() >= ((int64_t)1 << 20)) {
    try {
      th = std::thread(cand0);
    } catch (const std::system_error&) {
      cand0();  // no thread to be had: in turn
    }
  } else {
    cand0();
  }
  struct Join {  // candidate 0 finishes before this function returns or throws
    std::thread& t;
    ~Join() {
      if (t.joinable()) t.join();
    }
  } join{th};
  std::vector<int64_t> cand;
  int64_t nd1 = 0;
  bool have1 = false;
  {
    // Schur pattern on R = x u zero rows u auxiliary rows (local ids: x j -> j, zero
    // row r -> n + r, auxiliary row r -> n + mz + (r - ab))
    const int64_t R = n + mz + na;
    auto local = [&](int64_t u) -> int64_t {
      if (u < n || u - n < mz) return u;
      return (u - n >= ab) ? n + mz + (u - n - ab) : -1;
    };
    std::vector<std::vector<int64_t>> adj(R);
    for (int64_t u = 0; u < N; ++u) {
      const int64_t lu = local(u);
      if (lu < 0) continue;
      for (int64_t p = aptr[u]; p < aptr[u + 1]; ++p) {
        const int64_t lv = local(aidx[p]);
        if (lv >= 0) adj[lu].push_back(lv);
      }
    }
    // one clique per H block over its x neighbours
    int64_t pairs = 0;
    const int64_t pair_cap = 64 * (int64_t)aidx.size() + 50'000'000;
    bool dense = false;
    std::vector<int64_t> nb;
    std::vector<int64_t> mark(n, -1);
    for (size_t ci = 0; ci < hp.cl.cones.size() && !dense; ++ci) {
      const Cone& c = hp.cl.cones[ci];
      if (c.type == CLR_ZERO) continue;
      // each nonneg row, and each row of an expanded SOC, is its own 1x1 block
      const bool rowwise = c.type == CLR_NONNEG || c.aux >= 0;
      const int64_t nblk = rowwise ? c.dim : 1, bdim = rowwise ? 1 : c.dim;
      for (int64_t bk = 0; bk < nblk; ++bk) {
        nb.clear();
        if (c.aux >= 0) {  // the block's two auxiliary rows join its clique
          nb.push_back(n + mz + (c.aux - ab));
          nb.push_back(n + mz + (c.aux + 1 - ab));
        }
        const int64_t tag = (int64_t)ci * (1LL << 32) + bk;
        for (int64_t r = c.off + bk * bdim; r < c.off + (bk + 1) * bdim; ++r)
          for (int64_t p = hp.A.ptr[r]; p < hp.A.ptr[r + 1]; ++p) {
            const int64_t j = hp.A.idx[p];
            if (mark[j] != tag) {
              mark[j] = tag;
              nb.push_back(j);
            }
          }
        pairs += (int64_t)nb.size() * (int64_t)nb.size();
        if (pairs > pair_cap) {  // too dense to be worth it
          dense = true;
          break;
        }
        for (int64_t a : nb)
          for (int64_t b2 : nb)
            if (a != b2) adj[a].push_back(b2);
      }
    }
    if (!dense) {
      std::vector<int64_t> sptr(R + 1, 0), sidx;
      for (int64_t u = 0; u < R; ++u) {
        std::vector<int64_t>& a = adj[u];
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
        sptr[u + 1] = sptr[u] + (int64_t)a.size();
      }
      sidx.reserve(sptr[R]);
      for (int64_t u = 0; u < R; ++u) {
        sidx.insert(sidx.end(), adj[u].begin(), adj[u].end());
        std::vector<int64_t>().swap(adj[u]);
      }
      std::vector<int64_t> rperm;
      amd_order(R, sptr, sidx, rperm, nd1);
      cand.reserve(N);
      for (int64_t r = mz; r < ab; ++r) cand.push_back(n + r);
      for (int64_t v : rperm) cand.push_back(v < n + mz ? v : n + ab + (v - n - mz));  // local ids -> KKT indices
      have1 = true;
    }
  }
  int64_t nz1 = 0;
  double f1 = 0;
  if (have1) factor_counts(N, aptr, aidx, cand, &nz1, &f1);
  if (th.joinable()) th.join();
  if (err0) std::rethrow_exception(err0);
  if (have1 && f1 < f0) {
    order.swap(cand);
    n_dense = nd1;
    *which = 1;
  }
  return CLR_OK;
}

int symbolic_analyze(int64_t N, const std::vector<int64_t>& colptr, const std::vector<int64_t>& rowidx,
                     const std::vector<int64_t>* user_order, Symbolic& sy, int relax_) {
  sy = Symbolic();
  sy.N = N;
  // ---- symmetric adjacency for the ordering ----
  std::vector<int64_t> aptr, aidx;
  build_adjacency(N, colptr, rowidx, aptr, aidx);
  std::vector<int64_t> order;
  if (user_order) {
    order = *user_order;
    if ((int64_t)order.size() != N) return CLR_E_DIM;
    std::vector<char> seen(N, 0);
    for (int64_t v : order) {
      if (v < 0 || v >= N || seen[v]) return CLR_E_INVALID;
      seen[v] = 1;
    }
  } else {
    amd_order(N, aptr, aidx, order, sy.n_dense);
  }
  std::vector<int64_t> iorder(N);
  for (int64_t k = 0; k < N; ++k) iorder[order[k]] = k;

  // ---- elimination tree of the permuted matrix (Liu, with path compression) ----
  // row lists: for position k, positions i < k adjacent to k
  std::vector<int64_t> parent(N, -1), anc(N, -1);
  for (int64_t k = 0; k < N; ++k) {
    const int64_t v = order[k];
    for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) {
      int64_t i = iorder[aidx[p]];
      if (i >= k) continue;
      // walk from i to the root of its current subtree, compressing the path to k
      while (i != -1 && i != k) {
        int64_t nxt = anc[i];
        anc[i] = k;
        if (nxt == -1) parent[i] = k;
        i = nxt;
      }
    }
  }
  // ---- postorder (iterative DFS, children in increasing order) ----
  std::vector<int64_t> head(N, -1), nextc(N, -1);
  for (int64_t j = N - 1; j >= 0; --j)
    if (parent[j] >= 0) {
      nextc[j] = head[parent[j]];
      head[parent[j]] = j;
    }
  std::vector<int64_t> post;
  post.reserve(N);
  std::vector<int64_t> stack;
  for (int64_t r = 0; r < N; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      int64_t top = stack.back();
      int64_t c = head[top];
      if (c != -1) {
        head[top] = nextc[c];
        stack.push_back(c);
      } else {
        post.push_back(top);
        stack.pop_back();
      }
    }
  }
  // relabel: new position t = postorder index of old position post[t]
  std::vector<int64_t> ipost(N);
  for (int64_t t = 0; t < N; ++t) ipost[post[t]] = t;
  sy.perm.resize(N);
  sy.iperm.resize(N);
  for (int64_t t = 0; t < N; ++t) sy.perm[t] = order[post[t]];
  for (int64_t t = 0; t < N; ++t) sy.iperm[sy.perm[t]] = t;
  std::vector<int64_t> par(N, -1);
  for (int64_t t = 0; t < N; ++t) par[t] = (parent[post[t]] >= 0) ? ipost[parent[post[t]]] : -1;

  // ---- column structures (positions), fundamental supernodes ----
  // struct(j) = {j} u {i > j : K(i, j) != 0} u union over children c of struct(c) \ {c}
  std::vector<std::vector<int64_t>> cs(N);
  std::vector<int64_t> cc(N, 0);
  std::vector<int64_t> mark(N, -1);
  std::vector<int64_t> sn_of(N, -1);
  std::vector<int64_t> sn_ptr;
  std::vector<std::vector<int64_t>> sn_rows;
  std::vector<std::vector<int64_t>> kids(N);
  for (int64_t t = 0; t < N; ++t)
    if (par[t] >= 0) kids[par[t]].push_back(t);
  for (int64_t j = 0; j < N; ++j) {
    std::vector<int64_t> s;
    s.push_back(j);
    mark[j] = j;
    const int64_t v = sy.perm[j];
    for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) {
      int64_t i = sy.iperm[aidx[p]];
      if (i > j && mark[i] != j) {
        mark[i] = j;
        s.push_back(i);
      }
    }
    for (int64_t c : kids[j]) {
      for (int64_t i : cs[c])
        if (i != c && mark[i] != j) {
          mark[i] = j;
          s.push_back(i);
        }
      std::vector<int64_t>().swap(cs[c]);
    }
    std::sort(s.begin(), s.end());
    cc[j] = (int64_t)s.size();
    // j continues the supernode of j-1 if j-1 is a child of j and struct(j-1) = {j-1} u struct(j).
    // Other children of j may exist: their update rows lie inside struct(j), hence inside the
    // front of the supernode, which is all the multifrontal extend-add needs.
    bool cont = (j > 0 && par[j - 1] == j && cc[j - 1] == cc[j] + 1);
    if (!cont) {
      sn_ptr.push_back(j);
      sn_rows.push_back(s);
    }
    sn_of[j] = (int64_t)sn_ptr.size() - 1;
    cs[j] = std::move(s);
    if (par[j] < 0) std::vector<int64_t>().swap(cs[j]);
  }
  // exact factor statistics (fundamental supernodes hold no explicit zeros)
  sn_ptr.push_back(N);
  {
    const int64_t nf = (int64_t)sn_rows.size();
    sy.flops = 0;
    sy.l_nnz_exact = 0;
    for (int64_t J = 0; J < nf; ++J) {
      const int64_t f = (int64_t)sn_rows[J].size(), c = sn_ptr[J + 1] - sn_ptr[J];
      sy.l_nnz_exact += c * (c + 1) / 2 + c * (f - c);
      for (int64_t k = 0; k < c; ++k) {
        const double below = (double)(f - k - 1);
        sy.flops += below * (below + 1.0) + below;  // rank-1 update of the lower triangle + scaling
      }
    }
  }
  // ---- relaxed amalgamation ----
  // A child supernode is merged into its parent when the explicit zeros this
  // adds stay small relative to the merged panel -- the relaxed-supernode rule
  // of Ashcraft and Grimes with the usual thresholds (always up to 4 columns,
  // 80% zeros up to 16, 10% up to 48, 5% beyond; level 2 doubles the column
  // thresholds to 8 / 32 / 96).  Any child may merge, not
  // only the one whose columns end right before the parent's: its columns are
  // moved to just before the parent's (a topological reordering of the
  // elimination tree, so the fill is unchanged), children with the largest
  // update blocks first.  A merged child's update rows are a subset of the
  // parent's rows, so the merged front holds the child's columns followed by
  // the parent's rows.  Fewer, wider fronts: no large extend-adds of thin
  // supernodes, less front memory, fewer levels, more dense work per launch.
  if (relax_ > 0) {
    const int64_t c1 = relax_ >= 2 ? 8 : 4, c2 = 4 * c1, c3 = 12 * c1;
    const int64_t nf = (int64_t)sn_rows.size();
    std::vector<int64_t> fpar(nf, -1);
    for (int64_t J = 0; J < nf; ++J) {
      const int64_t last = sn_ptr[J + 1] - 1;
      fpar[J] = (par[last] >= 0) ? sn_of[par[last]] : -1;
    }
    std::vector<std::vector<int64_t>> skids(nf);
    for (int64_t J = 0; J < nf; ++J)
      if (fpar[J] >= 0) skids[fpar[J]].push_back(J);
    std::vector<int64_t> gc(nf), gz(nf, 0), gf(nf);     // merged group of J: columns, zeros, rows
    std::vector<int64_t> into(nf, -1);                 // J merged into into[J]
    std::vector<std::vector<int64_t>> group(nf);       // fundamental supernodes of the group, column order
    std::vector<std::vector<int64_t>> gkids(nf);       // unmerged children of J's group
    for (int64_t J = 0; J < nf; ++J) {
      gc[J] = sn_ptr[J + 1] - sn_ptr[J];
      gf[J] = (int64_t)sn_rows[J].size();
      group[J].push_back(J);
    }
    for (int64_t P = 0; P < nf; ++P) {  // children before parents
      // candidates: the children of P's group, largest update first; when a
      // child merges, its own unmerged children become children of the group
      std::priority_queue<std::pair<int64_t, int64_t>> cand;  // (update rows, -index)
      for (int64_t J : skids[P]) cand.emplace(gf[J] - gc[J], -J);
      while (!cand.empty()) {
        const int64_t J = -cand.top().second;
        cand.pop();
        const int64_t rJ = gf[J] - gc[J];
        const int64_t c = gc[J] + gc[P], f = gc[J] + gf[P];
        const int64_t z = gz[J] + gz[P] + gc[J] * (gf[P] - rJ);
        const double tot = (double)c * (double)f - 0.5 * (double)c * (double)(c - 1);
        const double zr = (double)z / tot;
        const bool merge = c <= c1 || (c <= c2 && zr < 0.8) || (c <= c3 && zr < 0.1) || zr < 0.05;
        if (!merge) {
          gkids[P].push_back(J);  // stays a child of P's group
          continue;
        }
        into[J] = P;
        gc[P] = c;
        gf[P] = f;
        gz[P] = z;
        std::vector<int64_t> g = std::move(group[J]);  // the child's columns go first
        g.insert(g.end(), group[P].begin(), group[P].end());
        group[P] = std::move(g);
        for (int64_t K : gkids[J]) cand.emplace(gf[K] - gc[K], -K);  // now children of P's group
        std::vector<int64_t>().swap(gkids[J]);
      }
    }
    // representatives (groups not merged further), their tree and a postorder of it
    std::vector<int64_t> rep(nf);
    for (int64_t J = nf - 1; J >= 0; --J) rep[J] = (into[J] < 0) ? J : rep[into[J]];
    std::vector<int64_t> rhead(nf, -1), rnext(nf, -1);
    std::vector<int64_t> roots;
    for (int64_t J = nf - 1; J >= 0; --J) {
      if (into[J] >= 0) continue;
      const int64_t Pr = fpar[J] >= 0 ? rep[fpar[J]] : -1;
      if (Pr < 0) {
        roots.push_back(J);
      } else {
        rnext[J] = rhead[Pr];
        rhead[Pr] = J;
      }
    }
    std::reverse(roots.begin(), roots.end());
    std::vector<int64_t> rpost;
    std::vector<int64_t> stk;
    for (int64_t R0 : roots) {
      stk.push_back(R0);
      while (!stk.empty()) {
        const int64_t top = stk.back();
        const int64_t ch = rhead[top];
        if (ch != -1) {
          rhead[top] = rnext[ch];
          stk.push_back(ch);
        } else {
          rpost.push_back(top);
          stk.pop_back();
        }
      }
    }
    // new positions: groups in postorder, each group's supernodes in its column order
    std::vector<int64_t> newpos(N);
    std::vector<int64_t> new_ptr;
    new_ptr.reserve(rpost.size() + 1);
    int64_t next = 0;
    for (int64_t R : rpost) {
      new_ptr.push_back(next);
      for (int64_t J : group[R])
        for (int64_t col = sn_ptr[J]; col < sn_ptr[J + 1]; ++col) newpos[col] = next++;
    }
    new_ptr.push_back(N);
    std::vector<std::vector<int64_t>> new_rows(rpost.size());
    for (size_t t = 0; t < rpost.size(); ++t) {
      const int64_t R = rpost[t];
      std::vector<int64_t>& rows = new_rows[t];
      rows.reserve((size_t)gf[R]);
      for (int64_t col = new_ptr[t]; col < new_ptr[t + 1]; ++col) rows.push_back(col);
      const int64_t ownc = sn_ptr[R + 1] - sn_ptr[R];
      for (size_t k = (size_t)ownc; k < sn_rows[R].size(); ++k) rows.push_back(newpos[sn_rows[R][k]]);
      std::sort(rows.begin() + (new_ptr[t + 1] - new_ptr[t]), rows.end());
      std::vector<int64_t>().swap(sn_rows[R]);
    }
    // relabel the order and the column tree
    std::vector<int64_t> perm2(N), par2(N, -1);
    for (int64_t j = 0; j < N; ++j) perm2[newpos[j]] = sy.perm[j];
    for (int64_t j = 0; j < N; ++j) par2[newpos[j]] = par[j] >= 0 ? newpos[par[j]] : -1;
    sy.perm.swap(perm2);
    for (int64_t t = 0; t < N; ++t) sy.iperm[sy.perm[t]] = t;
    par.swap(par2);
    sn_ptr.swap(new_ptr);
    sn_rows.swap(new_rows);
    for (int64_t t = 0; t + 1 < (int64_t)sn_ptr.size(); ++t)
      for (int64_t col = sn_ptr[t]; col < sn_ptr[t + 1]; ++col) sn_of[col] = t;
  }
  sy.nsn = (int64_t)sn_rows.size();
  sy.sn_ptr = sn_ptr;
  sy.sn_parent.assign(sy.nsn, -1);
  for (int64_t J = 0; J < sy.nsn; ++J) {
    int64_t last = sn_ptr[J + 1] - 1;
    sy.sn_parent[J] = (par[last] >= 0) ? sn_of[par[last]] : -1;
  }
  // rows, pools, statistics
  sy.row_ptr.assign(sy.nsn + 1, 0);
  for (int64_t J = 0; J < sy.nsn; ++J) sy.row_ptr[J + 1] = sy.row_ptr[J] + (int64_t)sn_rows[J].size();
  sy.rows.resize(sy.row_ptr[sy.nsn]);
  sy.front_off.resize(sy.nsn + 1);
  sy.upd_off.resize(sy.nsn + 1);
  sy.front_off[0] = 0;
  sy.upd_off[0] = 0;
  sy.l_nnz = 0;
  sy.flops_stored = 0;
  sy.max_front = 0;
  for (int64_t J = 0; J < sy.nsn; ++J) {
    std::copy(sn_rows[J].begin(), sn_rows[J].end(), sy.rows.begin() + sy.row_ptr[J]);
    const int64_t f = (int64_t)sn_rows[J].size();
    const int64_t c = sn_ptr[J + 1] - sn_ptr[J];
    sy.front_off[J + 1] = sy.front_off[J] + f * f;
    sy.upd_off[J + 1] = sy.upd_off[J] + f;
    sy.l_nnz += c * (c + 1) / 2 + c * (f - c);
    for (int64_t k = 0; k < c; ++k) {
      const double below = (double)(f - k - 1);
      sy.flops_stored += below * (below + 1.0) + below;
    }
    sy.max_front = std::max(sy.max_front, f);
  }
  sy.pool = sy.front_off[sy.nsn];
  sy.upd_total = sy.upd_off[sy.nsn];
  // level schedule: level(J) = 0 for leaves, 1 + max(level(children)) otherwise
  std::vector<int64_t> lev(sy.nsn, 0);
  int64_t maxlev = 0;
  for (int64_t J = 0; J < sy.nsn; ++J) {
    int64_t P = sy.sn_parent[J];
    if (P >= 0) lev[P] = std::max(lev[P], lev[J] + 1);
    maxlev = std::max(maxlev, lev[J]);
  }
  sy.nlev = sy.nsn ? maxlev + 1 : 0;
  sy.lev_ptr.assign(sy.nlev + 1, 0);
  for (int64_t J = 0; J < sy.nsn; ++J) sy.lev_ptr[lev[J] + 1]++;
  for (int64_t l = 0; l < sy.nlev; ++l) sy.lev_ptr[l + 1] += sy.lev_ptr[l];
  sy.lev_sn.resize(sy.nsn);
  {
    std::vector<int64_t> next(sy.lev_ptr.begin(), sy.lev_ptr.end() - 1);
    for (int64_t J = 0; J < sy.nsn; ++J) sy.lev_sn[next[lev[J]]++] = J;
  }
  return CLR_OK;
}

namespace {
// fronts whose children contribute at least this many entries build their lists on
// several host threads
constexpr int64_t kParallelEntries = (int64_t)1 << 22;

int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h, 8u));
}

// fn(block, scratch) for blocks 0 .. nblk-1 on nthr threads (blocks handed out by a
// counter), each thread with its own scratch of the given size; the first exception
// is rethrown after all threads are done.
template <class F>
void for_blocks(int64_t nblk, int nthr, int64_t scratch, F&& fn) {
  if (nthr <= 1) {
    std::vector<int64_t> w((size_t)scratch);
    for (int64_t bk = 0; bk < nblk; ++bk) fn(bk, w);
    return;
  }
  std::atomic<int64_t> next{0};
  std::exception_ptr err;
  std::mutex mu;
  auto body = [&] {
    try {
      std::vector<int64_t> w((size_t)scratch);
      for (int64_t bk; (bk = next.fetch_add(1)) < nblk;) fn(bk, w);
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu);
      if (!err) err = std::current_exception();
      next.store(nblk);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthr; ++t) {
    try {
      th.emplace_back(body);
    } catch (const std::system_error&) {
      break;  // fewer threads
    }
  }
  body();
  for (std::thread& t : th) t.join();
  if (err) std::rethrow_exception(err);
}
}  // namespace

// Index maps for the numeric phase.
void build_numeric_maps(const Symbolic& sy, const std::vector<int64_t>& kcol_ptr, const std::vector<int64_t>& krow,
                        NumericMaps& mp, bool direct) {
  const int64_t N = sy.N;
  mp = NumericMaps();
  std::vector<int64_t> sn_of(N);
  for (int64_t J = 0; J < sy.nsn; ++J)
    for (int64_t c = sy.sn_ptr[J]; c < sy.sn_ptr[J + 1]; ++c) sn_of[c] = J;
  // local index of each row of a front, filled per front on demand
  std::vector<int64_t> loc(N, -1);
  auto set_loc = [&](int64_t J) {
    for (int64_t k = sy.row_ptr[J]; k < sy.row_ptr[J + 1]; ++k) loc[sy.rows[k]] = k - sy.row_ptr[J];
  };
  // ---- kval entry -> pool position ----
  // Entry (i, j) of the lower triangle of K lands in the front of the supernode that owns
  // column min(iperm[i], iperm[j]), at (local row of max(..), local column of min(..)).
  const int64_t nk = (int64_t)krow.size();
  mp.kdest.assign(nk, -1);
  for (int64_t j = 0; j < N; ++j)
    for (int64_t p = kcol_ptr[j]; p < kcol_ptr[j + 1]; ++p) {
      int64_t a = sy.iperm[krow[p]], b = sy.iperm[j];
      int64_t r = std::max(a, b), c = std::min(a, b);
      int64_t J = sn_of[c];
      const int64_t* rb = sy.rows.data() + sy.row_ptr[J];
      const int64_t* re = sy.rows.data() + sy.row_ptr[J + 1];
      int64_t lr = std::lower_bound(rb, re, r) - rb;
      int64_t lc = c - sy.sn_ptr[J];
      int64_t f = re - rb;
      mp.kdest[p] = sy.front_off[J] + lr + lc * f;
    }
  // diagonal positions: for position k, its pool slot (k, k)
  mp.diag_pos.resize(N);
  for (int64_t k = 0; k < N; ++k) {
    int64_t J = sn_of[k];
    int64_t f = sy.row_ptr[J + 1] - sy.row_ptr[J];
    int64_t lc = k - sy.sn_ptr[J];
    mp.diag_pos[k] = sy.front_off[J] + lc + lc * f;
  }
  // ---- extend-add (factor) and update-gather (solve) pull maps, level by level ----
  // Targets are grouped by level of the receiving front, then by front, then by position.
  // Sources of one target appear in the order of the children (postorder), so every sum is
  // taken in a fixed order.
  std::vector<std::vector<int64_t>> children(sy.nsn);
  for (int64_t J = 0; J < sy.nsn; ++J)
    if (sy.sn_parent[J] >= 0) children[sy.sn_parent[J]].push_back(J);
  mp.fa_lev_ptr.assign(sy.nlev + 1, 0);
  mp.sv_lev_ptr.assign(sy.nlev + 1, 0);
  mp.px_lev_ptr.assign(sy.nlev + 1, 0);
  mp.px_round_ptr.assign(1, 0);
  mp.rel_off.assign(sy.nsn, -1);
  // children pushed by relative indices: the (up to kMaxPush) largest update
  // blocks of each front with at least kPushRows rows
  constexpr int64_t kPushRows = 64, kMaxPush = 4;
  std::vector<std::vector<int64_t>> pushed(sy.nsn);
  std::vector<char> is_pushed(sy.nsn, 0);
  auto upd_rows = [&](int64_t J) { return (sy.row_ptr[J + 1] - sy.row_ptr[J]) - (sy.sn_ptr[J + 1] - sy.sn_ptr[J]); };
  for (int64_t P = 0; P < sy.nsn; ++P) {
    std::vector<int64_t> big;
    for (int64_t ch : children[P])
      if (upd_rows(ch) >= kPushRows) big.push_back(ch);
    std::stable_sort(big.begin(), big.end(), [&](int64_t a, int64_t b) { return upd_rows(a) > upd_rows(b); });
    if ((int64_t)big.size() > kMaxPush) big.resize(kMaxPush);
    for (int64_t ch : big) is_pushed[ch] = 1;
    pushed[P] = std::move(big);
  }
  std::vector<std::pair<int64_t, int64_t>> contrib, ctmp;  // (target, source)
  std::vector<int64_t> cnt;
  // fronts up to this many entries get their pull lists by direct placement
  constexpr int64_t kDirectTargets = (int64_t)1 << 26;
  // counting pass: stable reorder of v by key(target) in [0, nb)
  auto count_pass = [&](std::vector<std::pair<int64_t, int64_t>>& from, std::vector<std::pair<int64_t, int64_t>>& to,
                        int64_t nb, auto key) {
    cnt.assign(nb + 1, 0);
    for (const auto& x : from) ++cnt[key(x.first) + 1];
    for (int64_t k = 0; k < nb; ++k) cnt[k + 1] += cnt[k];
    to.resize(from.size());
    for (const auto& x : from) to[cnt[key(x.first)]++] = x;
  };
  // stable sort by target of targets base + la + lb fP (2-D) or base + la (1-D)
  auto sort_by_target = [&](std::vector<std::pair<int64_t, int64_t>>& v, int64_t base, int64_t fP, bool two_d) {
    if (v.size() < 2) return;
    if (!two_d) {
      count_pass(v, ctmp, fP, [&](int64_t t) { return t - base; });
      v.swap(ctmp);
      return;
    }
    count_pass(v, ctmp, fP, [&](int64_t t) { return (t - base) % fP; });
    count_pass(ctmp, v, fP, [&](int64_t t) { return (t - base) / fP; });
  };
  {
    // exact sizes of the source lists (the pulls), so they are filled without regrowth
    int64_t nfa = 0, nsv = 0;
    for (int64_t J = 0; J < sy.nsn; ++J) {
      if (sy.sn_parent[J] < 0) continue;
      const int64_t u = upd_rows(J);
      nsv += u;
      if (!is_pushed[J]) nfa += u * (u + 1) / 2;
    }
    mp.fa_src.reserve(nfa);
    mp.sv_src.reserve(nsv);
  }
  for (int64_t l = 0; l < sy.nlev; ++l) {
    int64_t rounds = 0;
    for (int64_t t = sy.lev_ptr[l]; t < sy.lev_ptr[l + 1]; ++t) rounds = std::max<int64_t>(rounds, (int64_t)pushed[sy.lev_sn[t]].size());
    for (int64_t k = 0; k < rounds; ++k) {
      for (int64_t t = sy.lev_ptr[l]; t < sy.lev_ptr[l + 1]; ++t) {
        const int64_t P = sy.lev_sn[t];
        if ((int64_t)pushed[P].size() > k) mp.px_child.push_back(pushed[P][k]);
      }
      mp.px_round_ptr.push_back((int64_t)mp.px_child.size());
    }
    mp.px_lev_ptr[l + 1] = mp.px_lev_ptr[l] + rounds;
    for (int64_t t = sy.lev_ptr[l]; t < sy.lev_ptr[l + 1]; ++t) {
      const int64_t P = sy.lev_sn[t];
      if (children[P].empty()) continue;
      set_loc(P);
      const int64_t fP = sy.row_ptr[P + 1] - sy.row_ptr[P];
      for (int64_t ch : pushed[P]) {
        const int64_t f = sy.row_ptr[ch + 1] - sy.row_ptr[ch];
        const int64_t c = sy.sn_ptr[ch + 1] - sy.sn_ptr[ch];
        const int64_t* rr = sy.rows.data() + sy.row_ptr[ch];
        mp.rel_off[ch] = (int64_t)mp.rel.size();
        for (int64_t a = c; a < f; ++a) mp.rel.push_back((int32_t)loc[rr[a]]);
      }
      // factor: U_c entries (a >= b) -> F_P(loc(row a), loc(row b)), for the children not pushed
      int64_t ne = 0;
      for (int64_t ch : children[P])
        if (!is_pushed[ch]) ne += upd_rows(ch) * (upd_rows(ch) + 1) / 2;
      // the direct path scans all fP^2 targets of the parent: taken when the
      // children's contributions are comparable to that (else the sorted pairs)
      if (direct && ne > 0 && fP * fP <= kDirectTargets && fP * fP <= 4 * ne) {
        // two passes straight into the lists: count the sources of every target of
        // P's front, then place each source at its target's next slot -- targets in
        // increasing order, each target's sources in child / column / row order, as
        // the sorted pairs below give them.  Done per block of kColBlock parent
        // columns (targets are column-major, so the blocks come in target order and
        // a target's sources all fall in its block), which keeps the counts and the
        // block's slice of the lists in cache; the blocks are independent, so large
        // fronts count and place them on several host threads (the lists do not
        // depend on how the blocks are shared out).
        constexpr int64_t kColBlock = 16;
        const int64_t nblk = (fP + kColBlock - 1) / kColBlock;
        // the update columns b of each child whose parent column loc[rr[b]] lies in
        // [c0, c1): loc is increasing along a child's rows, so a contiguous range
        auto each_in = [&](int64_t c0, int64_t c1, auto&& fn) {
          for (int64_t ch : children[P]) {
            if (is_pushed[ch]) continue;
            const int64_t f = sy.row_ptr[ch + 1] - sy.row_ptr[ch];
            const int64_t c = sy.sn_ptr[ch + 1] - sy.sn_ptr[ch];
            const int64_t* rr = sy.rows.data() + sy.row_ptr[ch];
            const int64_t* lo = std::partition_point(rr + c, rr + f, [&](int64_t r) { return loc[r] < c0; });
            const int64_t* hi = std::partition_point(lo, rr + f, [&](int64_t r) { return loc[r] < c1; });
            for (int64_t b = lo - rr; b < hi - rr; ++b) {
              const int64_t lb = loc[rr[b]] - c0;
              for (int64_t a = b; a < f; ++a) fn(loc[rr[a]] + lb * fP, sy.front_off[ch] + a + b * f);
            }
          }
        };
        // per block: its targets that have sources (block-local index) and their counts
        std::vector<std::vector<int32_t>> btgt(nblk);
        std::vector<std::vector<int64_t>> bcnt(nblk);
        std::vector<int64_t> bstart(nblk);
        const int nthr = ne >= kParallelEntries ? std::min<int>(host_threads(), (int)nblk) : 1;
        for_blocks(nblk, nthr, kColBlock * fP, [&](int64_t bk, std::vector<int64_t>& cnt) {
          const int64_t c0 = bk * kColBlock, c1 = std::min(fP, c0 + kColBlock), nb = (c1 - c0) * fP;
          std::fill(cnt.begin(), cnt.begin() + nb, 0);
          each_in(c0, c1, [&](int64_t t, int64_t) { ++cnt[t]; });
          for (int64_t t = 0; t < nb; ++t)
            if (cnt[t]) {
              btgt[bk].push_back((int32_t)t);
              bcnt[bk].push_back(cnt[t]);
            }
        });
        int64_t pos = (int64_t)mp.fa_src.size();
        for (int64_t bk = 0; bk < nblk; ++bk) {
          bstart[bk] = pos;
          for (size_t q = 0; q < btgt[bk].size(); ++q) {
            mp.fa_tgt.push_back(sy.front_off[P] + bk * kColBlock * fP + btgt[bk][q]);
            mp.fa_ptr.push_back(pos);
            pos += bcnt[bk][q];
          }
        }
        mp.fa_src.resize(pos);
        for_blocks(nblk, nthr, kColBlock * fP, [&](int64_t bk, std::vector<int64_t>& slot) {
          const int64_t c0 = bk * kColBlock, c1 = std::min(fP, c0 + kColBlock);
          int64_t p = bstart[bk];
          for (size_t q = 0; q < btgt[bk].size(); ++q) {
            slot[btgt[bk][q]] = p;
            p += bcnt[bk][q];
          }
          int64_t* out = mp.fa_src.data();
          each_in(c0, c1, [&](int64_t t, int64_t src) { out[slot[t]++] = src; });
          std::vector<int32_t>().swap(btgt[bk]);
          std::vector<int64_t>().swap(bcnt[bk]);
        });
      } else if (ne > 0) {
        contrib.clear();
        contrib.reserve(ne);
        for (int64_t ch : children[P]) {
          if (is_pushed[ch]) continue;
          const int64_t f = sy.row_ptr[ch + 1] - sy.row_ptr[ch];
          const int64_t c = sy.sn_ptr[ch + 1] - sy.sn_ptr[ch];
          const int64_t* rr = sy.rows.data() + sy.row_ptr[ch];
          for (int64_t b = c; b < f; ++b) {
            int64_t lb = loc[rr[b]];
            for (int64_t a = b; a < f; ++a) {
              int64_t la = loc[rr[a]];
              contrib.emplace_back(sy.front_off[P] + la + lb * fP, sy.front_off[ch] + a + b * f);
            }
          }
        }
        // stable sort by target: targets are positions (row la, column lb) of P's
        // fP x fP front, so two stable counting passes -- by row, then by column --
        // order them as a comparison sort would, equal targets in insertion order
        sort_by_target(contrib, sy.front_off[P], fP, true);
        for (size_t q = 0; q < contrib.size(); ++q) {
          if (q == 0 || contrib[q].first != contrib[q - 1].first) {
            mp.fa_tgt.push_back(contrib[q].first);
            mp.fa_ptr.push_back((int64_t)mp.fa_src.size());
          }
          mp.fa_src.push_back(contrib[q].second);
        }
      }
      // solve: update vector entries of child c (w slots c_c .. f_c-1) -> w slot loc(row) of P
      contrib.clear();
      for (int64_t ch : children[P]) {
        const int64_t f = sy.row_ptr[ch + 1] - sy.row_ptr[ch];
        const int64_t c = sy.sn_ptr[ch + 1] - sy.sn_ptr[ch];
        const int64_t* rr = sy.rows.data() + sy.row_ptr[ch];
        for (int64_t a = c; a < f; ++a) contrib.emplace_back(sy.upd_off[P] + loc[rr[a]], sy.upd_off[ch] + a);
      }
      sort_by_target(contrib, sy.upd_off[P], fP, false);  // targets: P's fP work slots
      for (size_t q = 0; q < contrib.size(); ++q) {
        if (q == 0 || contrib[q].first != contrib[q - 1].first) {
          mp.sv_tgt.push_back(contrib[q].first);
          mp.sv_ptr.push_back((int64_t)mp.sv_src.size());
        }
        mp.sv_src.push_back(contrib[q].second);
      }
    }
    mp.fa_lev_ptr[l + 1] = (int64_t)mp.fa_tgt.size();
    mp.sv_lev_ptr[l + 1] = (int64_t)mp.sv_tgt.size();
  }
  mp.fa_ptr.push_back((int64_t)mp.fa_src.size());
  mp.sv_ptr.push_back((int64_t)mp.sv_src.size());
  // KKT index of every front row (the solves read and write vectors in KKT order)
  mp.rows_kkt.resize(sy.rows.size());
  for (size_t k = 0; k < sy.rows.size(); ++k) mp.rows_kkt[k] = (int32_t)sy.perm[sy.rows[k]];
}

uint64_t maps_digest(const Symbolic& sy, const NumericMaps& mp) {
  // FNV-1a's step (xor, then multiply by the 64-bit FNV prime) applied to whole
  // entries rather than bytes: one multiply per index
  uint64_t h = 1469598103934665603ull;
  auto word = [&](uint64_t x) { h = (h ^ x) * 1099511628211ull; };
  auto add = [&](const auto& v) {
    word((uint64_t)v.size());
    for (const auto& x : v) word((uint64_t)(int64_t)x);
  };
  add(sy.perm);
  add(mp.kdest);
  add(mp.diag_pos);
  add(mp.fa_lev_ptr);
  add(mp.fa_tgt);
  add(mp.fa_ptr);
  add(mp.fa_src);
  add(mp.px_lev_ptr);
  add(mp.px_round_ptr);
  add(mp.px_child);
  add(mp.rel_off);
  add(mp.rel);
  add(mp.sv_lev_ptr);
  add(mp.sv_tgt);
  add(mp.sv_ptr);
  add(mp.sv_src);
  add(mp.rows_kkt);
  return h;
}

}  // namespace clr
