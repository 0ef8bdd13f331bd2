// Oracle for the halo-finding path: a plain, slow, single-node-at-a-time CPU restatement of
// 3D friends-of-friends, the recursive 6D phase-space FoF hierarchy, potential-based unbinding
// and halo properties.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path calls this code: only the tests, the
// smoke check and the benchmark's CPU-baseline leg load it. It shares no code, header, table or
// helper with the CUDA library.
//
// What the paper fixes: each process runs 3D FoF on its particles, then finds subhalos inside
// every FoF halo from 6D phase-space information (Section "Parallelization"), and the halo
// catalogue carries extra properties such as the inertia tensor (Summary). The linking length
// b = 0.28, the 6D metric |dx|^2/sx^2 + |dv|^2/sv^2, the linked fraction f = 0.7 with recursion,
// the 0.5 bound-fraction threshold and the 10-particle minimum are Rockstar's parameters
// (Behroozi et al. 2013, cited in the Summary). Every rounding-level choice below (operation
// order, <= vs <, the canonical FP64 reduction order) is a reading this implementation fixes so
// that a GPU implementation can reproduce it bit for bit.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread
// (-ffp-contract=off matters on aarch64, where GCC contracts a*b+c into FMA by default.)

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <numeric>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Periodic minimum-image difference of two float32 coordinates (3D FoF, Section
// "Parallelization"): d = b - a rounded to float32; if d > L/2 subtract L, else if d < -L/2 add L.
// IEEE round-to-nearest commutes with negation, so wrap(b - a) == -wrap(a - b) exactly.
inline float wrap_diff(float a, float b, float L, float hL) {
  float d = b - a;
  if (d > hL) {
    d = d - L;
  } else if (d < -hL) {
    d = d + L;
  }
  return d;
}

// Squared distance, float32, left to right, no fused multiply-add: (dx*dx + dy*dy) + dz*dz.
inline float sq3(float dx, float dy, float dz) {
  float a = dx * dx;
  float b = dy * dy;
  float c = dz * dz;
  float s = a + b;
  return s + c;
}

// Plain union-find with path halving; roots are the smallest index of their set.
struct UnionFind {
  std::vector<int64_t> p;
  explicit UnionFind(int64_t n) : p(n) { std::iota(p.begin(), p.end(), int64_t(0)); }
  int64_t find(int64_t x) {
    while (p[x] != x) {
      p[x] = p[p[x]];
      x = p[x];
    }
    return x;
  }
  void unite(int64_t a, int64_t b) {
    a = find(a);
    b = find(b);
    if (a == b) return;
    if (a < b) p[b] = a; else p[a] = b;
  }
};

// ---------------------------------------------------------------------------------------------
// Canonical reduction order (CRO) for every FP64 sum of the path. For a[0..m):
//   chunks of 1024 consecutive terms; inside chunk c, lane l (0..31) sums a[1024c + l + 32k]
//   for k = 0..31 in order, starting from 0.0; lanes are then combined by halving,
//   s[l] = s[l] + s[l + off] for off = 16, 8, 4, 2, 1; the chunk total is s[0]. Chunk totals
//   are combined by a pairwise tree, t'[k] = t[2k] + t[2k+1], an odd last element carried up.
// An empty sequence sums to 0.0.
template <class Term>
double cro_sum(int64_t m, Term term) {
  if (m <= 0) return 0.0;
  const int64_t chunks = (m + 1023) / 1024;
  std::vector<double> t(chunks);
  for (int64_t c = 0; c < chunks; ++c) {
    double s[32];
    for (int l = 0; l < 32; ++l) {
      double acc = 0.0;
      for (int k = 0; k < 32; ++k) {
        const int64_t idx = c * 1024 + l + 32 * k;
        if (idx < m) acc = acc + term(idx);
      }
      s[l] = acc;
    }
    for (int off = 16; off >= 1; off >>= 1)
      for (int l = 0; l < off; ++l) s[l] = s[l] + s[l + off];
    t[c] = s[0];
  }
  while (t.size() > 1) {
    std::vector<double> nt;
    nt.reserve((t.size() + 1) / 2);
    for (size_t k = 0; 2 * k + 1 < t.size(); ++k) nt.push_back(t[2 * k] + t[2 * k + 1]);
    if (t.size() % 2 == 1) nt.push_back(t.back());
    t.swap(nt);
  }
  return t[0];
}

// Run f(i) for i in [0, count) on up to `threads` std::threads (static interleaved split).
template <class F>
void parallel_for(int64_t count, int threads, F f) {
  if (threads <= 1 || count <= 1) {
    for (int64_t i = 0; i < count; ++i) f(i);
    return;
  }
  const int nt = int(std::min<int64_t>(threads, count));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([=]() {
      for (int64_t i = t; i < count; i += nt) f(i);
    });
  for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------------------------------------
// 3D FoF link predicate: i ~ j iff the float32 periodic squared distance is <= ll^2 (float32).
inline bool fof_linked(const float* pos, int64_t i, int64_t j, float L, float hL, float ll2) {
  const float dx = wrap_diff(pos[3 * i + 0], pos[3 * j + 0], L, hL);
  const float dy = wrap_diff(pos[3 * i + 1], pos[3 * j + 1], L, hL);
  const float dz = wrap_diff(pos[3 * i + 2], pos[3 * j + 2], L, hL);
  return sq3(dx, dy, dz) <= ll2;
}

// Labels = smallest id in each connected component of the link graph.
void labels_from_uf(int64_t n, const int64_t* ids, UnionFind& uf, int64_t* labels) {
  std::vector<int64_t> min_id(n, INT64_MAX);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t r = uf.find(i);
    min_id[r] = std::min(min_id[r], ids[i]);
  }
  for (int64_t i = 0; i < n; ++i) labels[i] = min_id[uf.find(i)];
}

// ---------------------------------------------------------------------------------------------
// 6D phase-space hierarchy (Section "Parallelization": subhalo finding per FoF halo from 6D
// phase-space information).
struct Node {
  int64_t parent;
  int32_t level;
  int64_t min_id;
  int64_t size;
  int64_t off;  // into the member list
  float scal[3] = {0.f, 0.f, 0.f};  // inv_sx2, inv_sv2, l2 of the node's split
};

struct Hierarchy {
  int64_t n = 0;
  std::vector<Node> nodes;
  std::vector<int64_t> members;  // particle indices; each node's members in ascending id order
  std::vector<int64_t> deepest;  // per particle: deepest node holding it, -1 if none
};

// Positions of a node's members relative to its reference member (the smallest id), float32.
void unwrap_node(const float* pos, const int64_t* mem, int64_t g, float L, std::vector<float>& u) {
  const float hL = 0.5f * L;
  const int64_t r = mem[0];
  u.resize(3 * g);
  for (int64_t a = 0; a < g; ++a)
    for (int d = 0; d < 3; ++d) u[3 * a + d] = wrap_diff(pos[3 * r + d], pos[3 * mem[a] + d], L, hL);
}

// Total (3-dimension) variance of a float32 [g][3] array from CRO FP64 moments:
// mean_d = S_d / g; var = ((Q_0/g - mean_0^2) + (Q_1/g - mean_1^2)) + (Q_2/g - mean_2^2).
double total_variance(const float* a, int64_t g) {
  double var = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double s = cro_sum(g, [&](int64_t i) { return double(a[3 * i + d]); });
    const double q = cro_sum(g, [&](int64_t i) { return double(a[3 * i + d]) * double(a[3 * i + d]); });
    const double mean = s / double(g);
    const double term = q / double(g) - mean * mean;
    var = (d == 0) ? term : var + term;
  }
  return var;
}

inline float inv_or_zero(double var) { return var > 0.0 ? float(1.0 / var) : 0.0f; }

// 6D squared distance, float32, no FMA:
// fl(fl(|du|^2) * inv_sx2) + fl(fl(|dv|^2) * inv_sv2), |d|^2 = (dx*dx + dy*dy) + dz*dz.
inline float d6(const float* u, const float* v, int64_t i, int64_t j, float isx, float isv) {
  const float rx = sq3(u[3 * j] - u[3 * i], u[3 * j + 1] - u[3 * i + 1], u[3 * j + 2] - u[3 * i + 2]);
  const float rv = sq3(v[3 * j] - v[3 * i], v[3 * j + 1] - v[3 * i + 1], v[3 * j + 2] - v[3 * i + 2]);
  const float a = rx * isx;
  const float b = rv * isv;
  return a + b;
}

struct SplitResult {
  float inv_sx2 = 0.f, inv_sv2 = 0.f, l2 = 0.f;
  std::vector<float> nn2;
  std::vector<int64_t> comp;  // per member: smallest member position of its 6D component
};

// ---------------------------------------------------------------------------------------------
// Exactly pruned 6D searches for large nodes: the same nearest-neighbour distances and the
// same link graph as the all-pairs loops, found with a k-d tree. Points are scaled into the
// space where the plain squared Euclidean distance is the 6D metric,
// P = (u sqrt(inv_sx2), v sqrt(inv_sv2)) in float64. The float32 d6 of the definition is a
// handful of correctly rounded operations away from that exact distance (relative error below
// 1e-6), so a tree cell whose float64 lower bound exceeds (1 + 1e-5) times the current best
// (or l2), plus 1e-30 for underflow, cannot hold a member whose float32 d6 is at most the best:
// pruning never removes the minimum or a link, and every value used is the definition's float32
// d6. Cells are split at the median of their widest coordinate down to 16 points.
struct KdTree {
  struct Cell {
    double lo[6], hi[6];
    int64_t a, b;             // point range [a, b) in idx
    int64_t left = -1, right = -1;
  };
  std::vector<double> P;      // [g][6]
  std::vector<int64_t> idx;   // point order
  std::vector<Cell> cells;

  KdTree(const float* u, const float* v, int64_t g, float isx, float isv) : P(6 * g), idx(g) {
    const double sx = std::sqrt(double(isx)), sv = std::sqrt(double(isv));
    for (int64_t i = 0; i < g; ++i) {
      for (int d = 0; d < 3; ++d) {
        P[6 * i + d] = double(u[3 * i + d]) * sx;
        P[6 * i + 3 + d] = double(v[3 * i + d]) * sv;
      }
      idx[i] = i;
    }
    cells.reserve(size_t(2 * (g / 8 + 1)));
    build(0, g);
  }

  int64_t build(int64_t a, int64_t b) {
    Cell c;
    c.a = a;
    c.b = b;
    for (int d = 0; d < 6; ++d) {
      c.lo[d] = INFINITY;
      c.hi[d] = -INFINITY;
    }
    for (int64_t k = a; k < b; ++k)
      for (int d = 0; d < 6; ++d) {
        c.lo[d] = std::min(c.lo[d], P[6 * idx[k] + d]);
        c.hi[d] = std::max(c.hi[d], P[6 * idx[k] + d]);
      }
    const int64_t id = int64_t(cells.size());
    cells.push_back(c);
    if (b - a > 16) {
      int w = 0;
      for (int d = 1; d < 6; ++d)
        if (c.hi[d] - c.lo[d] > c.hi[w] - c.lo[w]) w = d;
      const int64_t mid = a + (b - a) / 2;
      std::nth_element(idx.begin() + a, idx.begin() + mid, idx.begin() + b,
                       [&](int64_t x, int64_t y) { return P[6 * x + w] < P[6 * y + w]; });
      const int64_t l = build(a, mid);
      const int64_t r = build(mid, b);
      cells[id].left = l;
      cells[id].right = r;
    }
    return id;
  }

  double lower_bound(int64_t c, int64_t i) const {
    double s = 0.0;
    for (int d = 0; d < 6; ++d) {
      const double x = P[6 * i + d];
      const double gap = x < cells[c].lo[d] ? cells[c].lo[d] - x
                                            : (x > cells[c].hi[d] ? x - cells[c].hi[d] : 0.0);
      s += gap * gap;
    }
    return s;
  }

  // Visit every point j of the cells whose lower bound from point i is at most
  // *limit (1 + 1e-5) + 1e-30; *limit is re-read before each cell, so a shrinking best prunes more.
  template <class Visit>
  void search(int64_t i, const float* limit, Visit visit) const {
    std::vector<int64_t> stack{0};
    while (!stack.empty()) {
      const int64_t c = stack.back();
      stack.pop_back();
      if (lower_bound(c, i) > double(*limit) * (1.0 + 1e-5) + 1e-30) continue;
      if (cells[c].left < 0) {
        for (int64_t k = cells[c].a; k < cells[c].b; ++k) visit(idx[k]);
        continue;
      }
      const int64_t l = cells[c].left, r = cells[c].right;
      if (lower_bound(l, i) <= lower_bound(r, i)) {  // nearer child on top of the stack
        stack.push_back(r);
        stack.push_back(l);
      } else {
        stack.push_back(l);
        stack.push_back(r);
      }
    }
  }
};

// Nodes above this size use the pruned searches, with their members spread over threads.
constexpr int64_t kPrunedMin = 4096;

// One level of 6D FoF on a node whose members (ascending id) have unwrapped positions u and
// velocities v: sigma from CRO moments, nearest-neighbour distances, the adaptive link length
// (the k-th smallest nn2 with k = ceil(f g) - 1), and the components of the link graph. All
// pairs when g <= kPrunedMin (pruned < 0) or pruned == 0, the k-d tree otherwise.
void split_node(const float* u, const float* v, int64_t g, int32_t f_num, int32_t f_den,
                SplitResult& out, int threads = 1, int pruned = -1) {
  out.inv_sx2 = inv_or_zero(total_variance(u, g));
  out.inv_sv2 = inv_or_zero(total_variance(v, g));
  out.nn2.assign(g, INFINITY);
  const bool use_tree = pruned < 0 ? g > kPrunedMin : pruned != 0;
  const int64_t k = (int64_t(f_num) * g + f_den - 1) / f_den - 1;
  UnionFind uf(g);
  if (!use_tree) {
    for (int64_t i = 0; i < g; ++i) {
      float best = INFINITY;
      for (int64_t j = 0; j < g; ++j) {
        if (j == i) continue;
        const float d = d6(u, v, i, j, out.inv_sx2, out.inv_sv2);
        if (d < best) best = d;
      }
      out.nn2[i] = best;
    }
    std::vector<float> sorted(out.nn2);
    std::nth_element(sorted.begin(), sorted.begin() + k, sorted.end());
    out.l2 = sorted[k];
    for (int64_t i = 0; i < g; ++i)
      for (int64_t j = i + 1; j < g; ++j)
        if (d6(u, v, i, j, out.inv_sx2, out.inv_sv2) <= out.l2) uf.unite(i, j);
  } else {
    const KdTree tree(u, v, g, out.inv_sx2, out.inv_sv2);
    parallel_for(g, threads, [&](int64_t i) {
      float best = INFINITY;
      tree.search(i, &best, [&](int64_t j) {
        if (j == i) return;
        const float d = d6(u, v, i, j, out.inv_sx2, out.inv_sv2);
        if (d < best) best = d;
      });
      out.nn2[i] = best;
    });
    std::vector<float> sorted(out.nn2);
    std::nth_element(sorted.begin(), sorted.begin() + k, sorted.end());
    out.l2 = sorted[k];
    // link pairs (i < j) collected per thread, then united in one thread
    const int nt = int(std::max<int64_t>(1, std::min<int64_t>(threads, g)));
    std::vector<std::vector<std::pair<int64_t, int64_t>>> edges(nt);
    const float l2 = out.l2;
    parallel_for(nt, nt, [&](int64_t t) {
      for (int64_t i = t; i < g; i += nt) {
        if (out.nn2[i] > l2) continue;  // no other member is within l2
        tree.search(i, &l2, [&](int64_t j) {
          if (j > i && d6(u, v, i, j, out.inv_sx2, out.inv_sv2) <= l2) edges[t].emplace_back(i, j);
        });
      }
    });
    for (auto& e : edges)
      for (auto& pr : e) uf.unite(pr.first, pr.second);
  }
  out.comp.resize(g);
  for (int64_t i = 0; i < g; ++i) out.comp[i] = uf.find(i);
}

// Children of a split node: components with at least min_size members and fewer than g.
// Returned in ascending order of their smallest member (hence of their min id); each child's
// member positions ascend.
std::vector<std::vector<int64_t>> children_of(const SplitResult& s, int64_t g, int32_t min_size) {
  std::vector<int64_t> count(g, 0);
  for (int64_t i = 0; i < g; ++i) count[s.comp[i]]++;
  std::vector<int64_t> slot(g, -1);
  std::vector<std::vector<int64_t>> kids;
  for (int64_t i = 0; i < g; ++i) {
    const int64_t c = s.comp[i];
    if (count[c] < min_size || count[c] >= g) continue;
    if (slot[c] < 0) {
      slot[c] = int64_t(kids.size());
      kids.emplace_back();
    }
    kids[slot[c]].push_back(i);
  }
  return kids;
}

Hierarchy* build_hierarchy(int64_t n, const float* pos, const float* vel, const int64_t* ids,
                           const int64_t* fof_label, float L, int32_t f_num, int32_t f_den,
                           int32_t min_size, int threads) {
  auto* h = new Hierarchy();
  h->n = n;
  h->deepest.assign(n, -1);
  // Level 0: FoF groups with at least min_size particles, by ascending label (= min id); members
  // by ascending id.
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), int64_t(0));
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return fof_label[a] != fof_label[b] ? fof_label[a] < fof_label[b] : ids[a] < ids[b];
  });
  for (int64_t s = 0; s < n;) {
    int64_t e = s;
    while (e < n && fof_label[order[e]] == fof_label[order[s]]) ++e;
    if (e - s >= min_size) {
      Node nd{-1, 0, ids[order[s]], e - s, int64_t(h->members.size())};
      h->nodes.push_back(nd);
      h->members.insert(h->members.end(), order.begin() + s, order.begin() + e);
    }
    s = e;
  }
  // Breadth-first: split every node of a level (independently, possibly in parallel), then
  // append the children in (parent, min id) order. Levels therefore appear in order.
  int64_t level_begin = 0;
  int32_t level = 0;
  while (level_begin < int64_t(h->nodes.size())) {
    const int64_t level_end = int64_t(h->nodes.size());
    const int64_t count = level_end - level_begin;
    std::vector<std::vector<std::vector<int64_t>>> kids(count);
    auto split_one = [&](int64_t q, int inner_threads) {
      const Node nd = h->nodes[level_begin + q];
      const int64_t* mem = h->members.data() + nd.off;
      std::vector<float> u, v(3 * nd.size);
      unwrap_node(pos, mem, nd.size, L, u);
      for (int64_t a = 0; a < nd.size; ++a)
        for (int d = 0; d < 3; ++d) v[3 * a + d] = vel[3 * mem[a] + d];
      SplitResult sr;
      split_node(u.data(), v.data(), nd.size, f_num, f_den, sr, inner_threads);
      kids[q] = children_of(sr, nd.size, min_size);
      float* sc = h->nodes[level_begin + q].scal;
      sc[0] = sr.inv_sx2;
      sc[1] = sr.inv_sv2;
      sc[2] = sr.l2;
    };
    // small nodes: one per thread; large nodes one after another, each over all threads
    parallel_for(count, threads, [&](int64_t q) {
      if (h->nodes[level_begin + q].size <= kPrunedMin) split_one(q, 1);
    });
    for (int64_t q = 0; q < count; ++q)
      if (h->nodes[level_begin + q].size > kPrunedMin) split_one(q, threads);
    for (int64_t q = 0; q < count; ++q) {
      const int64_t parent = level_begin + q;
      for (auto& kid : kids[q]) {
        const Node pn = h->nodes[parent];
        Node nd{parent, level + 1, ids[h->members[pn.off + kid[0]]], int64_t(kid.size()),
                int64_t(h->members.size())};
        for (int64_t a : kid) h->members.push_back(h->members[pn.off + a]);
        h->nodes.push_back(nd);
      }
    }
    level_begin = level_end;
    ++level;
  }
  for (int64_t q = 0; q < int64_t(h->nodes.size()); ++q)
    for (int64_t a = 0; a < h->nodes[q].size; ++a) h->deepest[h->members[h->nodes[q].off + a]] = q;
  return h;
}

// Bulk velocity of a node: CRO(v_d) / g per axis.
void bulk_velocity(const float* vel, const int64_t* mem, int64_t g, double* vb) {
  for (int d = 0; d < 3; ++d)
    vb[d] = cro_sum(g, [&](int64_t a) { return double(vel[3 * mem[a] + d]); }) / double(g);
}

// Potential and flag of member i of a node (unwrapped positions u, bulk velocity vb; members j
// with in[j] == 0 contribute 0.0 when the mask `in` is given):
//   phi_i = -(G m) CRO_j( j == i ? 0 : 1 / sqrt(((Dx Dx + Dy Dy) + Dz Dz) + eps^2) ),
//   D = (double)u_j - (double)u_i; KE_i = 0.5 ((dvx dvx + dvy dvy) + dvz dvz),
//   dv = (double)v_i - vb; bound iff KE_i + phi_i < 0.
bool member_energy(const float* u, const float* vel, const int64_t* mem, int64_t g, int64_t i,
                   const double* vb, double eps2, double Gm, double* phi_out,
                   const uint8_t* in = nullptr) {
  const double s = cro_sum(g, [&](int64_t j) {
    if (j == i || (in && !in[j])) return 0.0;
    const double dx = double(u[3 * j]) - double(u[3 * i]);
    const double dy = double(u[3 * j + 1]) - double(u[3 * i + 1]);
    const double dz = double(u[3 * j + 2]) - double(u[3 * i + 2]);
    const double r2 = (dx * dx + dy * dy) + dz * dz;
    return 1.0 / std::sqrt(r2 + eps2);
  });
  const double p = -(Gm * s);
  const double dvx = double(vel[3 * mem[i]]) - vb[0];
  const double dvy = double(vel[3 * mem[i] + 1]) - vb[1];
  const double dvz = double(vel[3 * mem[i] + 2]) - vb[2];
  const double ke = 0.5 * ((dvx * dvx + dvy * dvy) + dvz * dvz);
  *phi_out = p;
  return (ke + p) < 0.0;
}

// Seed halos and their particles (the step after the 6D hierarchy; the paper names it only as
// subhalo finding inside every FoF halo, so this is a stated reading):
//   seeds: the nodes without children (every level-0 node has at least one under it);
//   frame: u = C1-wrapped offset from the level-0 node's reference member r0 (its smallest id);
//   seed s: centre c_s = float(double(wrap(x_{r_s} - x_{r0})) + CRO(u^s) / g_s) with u^s the
//     offsets from s's own reference member r_s, bulk velocity w_s = float(CRO(v) / g_s), and
//     the metric scales inv_sx2_s, inv_sv2_s of s's own 6D split;
//   distance to a seed: fl(|u - c_s|^2 inv_sx2_s) + fl(|v - w_s|^2 inv_sv2_s), float32 in d6's
//     operation order;
//   particle: the seed holding it when its deepest node is a seed, otherwise the nearest seed
//     under its deepest node (ties: the smaller node index);
//   host of a seed s: among the other seeds of the same level-0 node that rank above it (more
//     assigned particles; equal counts: the smaller node index ranks above), the nearest by the
//     candidate's metric evaluated at (c_s, w_s); -1 if none ranks above.
// Outputs: particle_seed [n] (-1 outside every node), node_host [n_nodes] (-2 for a node that is
// not a seed), node_count [n_nodes] (particles assigned; 0 for a node that is not a seed).
inline float metric6(const float* a, const float* b, const float* va, const float* vb, float isx,
                     float isv) {
  const float rx = sq3(a[0] - b[0], a[1] - b[1], a[2] - b[2]);
  const float rv = sq3(va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]);
  const float x = rx * isx;
  const float y = rv * isv;
  return x + y;
}

int assign_seeds(int64_t n, const float* pos, const float* vel, float L, int64_t nn,
                 const int64_t* parent, const int64_t* member_off, const int64_t* member_idx,
                 const int64_t* deepest, const float* params, int threads, int64_t* particle_seed,
                 int64_t* node_host, int64_t* node_count) {
  const float hL = 0.5f * L;
  std::vector<int64_t> nkids(nn, 0), root(nn);
  for (int64_t q = 0; q < nn; ++q) {
    if (parent[q] >= 0) nkids[parent[q]]++;
    root[q] = parent[q] < 0 ? q : root[parent[q]];  // parents precede their children
  }
  std::vector<float> cen(3 * nn, 0.f), bulk(3 * nn, 0.f);
  std::vector<std::vector<int64_t>> under(nn);  // seeds under each node, ascending index
  for (int64_t s = 0; s < nn; ++s) {
    node_host[s] = -2;
    node_count[s] = 0;
    if (nkids[s] != 0) continue;
    const int64_t g = member_off[s + 1] - member_off[s];
    const int64_t* mem = member_idx + member_off[s];
    const int64_t rs = mem[0], r0 = member_idx[member_off[root[s]]];
    std::vector<float> u;
    unwrap_node(pos, mem, g, L, u);
    for (int d = 0; d < 3; ++d) {
      const float o = wrap_diff(pos[3 * r0 + d], pos[3 * rs + d], L, hL);
      const double su = cro_sum(g, [&](int64_t a) { return double(u[3 * a + d]); });
      const double sv = cro_sum(g, [&](int64_t a) { return double(vel[3 * mem[a] + d]); });
      cen[3 * s + d] = float(double(o) + su / double(g));
      bulk[3 * s + d] = float(sv / double(g));
    }
    for (int64_t q = s; q >= 0; q = parent[q]) under[q].push_back(s);
  }
  for (auto& v : under) std::sort(v.begin(), v.end());
  for (int64_t i = 0; i < n; ++i) particle_seed[i] = -1;
  parallel_for(n, threads, [&](int64_t i) {
    const int64_t dq = deepest[i];
    if (dq < 0) return;
    if (nkids[dq] == 0) {
      particle_seed[i] = dq;
      return;
    }
    const int64_t r0 = member_idx[member_off[root[dq]]];
    float u[3];
    for (int d = 0; d < 3; ++d) u[d] = wrap_diff(pos[3 * r0 + d], pos[3 * i + d], L, hL);
    float best = INFINITY;
    int64_t arg = -1;
    for (int64_t s : under[dq]) {
      const float d = metric6(u, &cen[3 * s], vel + 3 * i, &bulk[3 * s], params[3 * s], params[3 * s + 1]);
      if (arg < 0 || d < best) {
        best = d;
        arg = s;
      }
    }
    particle_seed[i] = arg;
  });
  for (int64_t i = 0; i < n; ++i)
    if (particle_seed[i] >= 0) node_count[particle_seed[i]]++;
  for (int64_t s = 0; s < nn; ++s) {
    if (nkids[s] != 0) continue;
    float best = INFINITY;
    int64_t arg = -1;
    for (int64_t h : under[root[s]]) {
      if (h == s) continue;
      const bool above = node_count[h] > node_count[s] || (node_count[h] == node_count[s] && h < s);
      if (!above) continue;
      const float d = metric6(&cen[3 * s], &cen[3 * h], &bulk[3 * s], &bulk[3 * h], params[3 * h],
                              params[3 * h + 1]);
      if (arg < 0 || d < best) {
        best = d;
        arg = h;
      }
    }
    node_host[s] = arg;
  }
  return 0;
}

}  // namespace

// =============================================================================================
// C ABI (ctypes). Every array is host memory owned by the caller; positions/velocities are
// float32 [n][3], ids int64 [n]. Functions return 0 on success, -1 on invalid arguments.
extern "C" {

int or_split_node_ex(int64_t g, const float* u, const float* v, int32_t f_num, int32_t f_den,
                     int32_t pruned, int32_t threads, float* scal_out, float* nn2_out,
                     int64_t* comp_out);
int or_unbind_iter(int64_t n_nodes, const int64_t* member_off, const int64_t* member_idx,
                   const float* pos, const float* vel, float L, float eps, double G, double m,
                   int32_t min_size, int32_t bf_num, int32_t bf_den, int32_t passes,
                   int32_t threads, double* phi, uint8_t* bound, int64_t* n_bound,
                   uint8_t* is_halo, double* m_bound);

// Brute-force 3D FoF over all pairs: labels[i] = smallest id of i's component.
int or_fof3d_brute(int64_t n, const float* pos, const int64_t* ids, float L, float ll,
                   int64_t* labels) {
  if (n < 0 || (n > 0 && (!pos || !ids || !labels))) return -1;
  const float hL = 0.5f * L, ll2 = ll * ll;
  UnionFind uf(n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j)
      if (fof_linked(pos, i, j, L, hL, ll2)) uf.unite(i, j);
  labels_from_uf(n, ids, uf, labels);
  return 0;
}

// 3D FoF with a cell grid: cells of side L/nc >= 1.01 ll, so any linked pair lies in the same or
// adjacent (periodic) cells; each pair of candidate particles is tested with the same predicate
// as the brute-force version. Cell coordinates are computed in float64.
int or_fof3d_grid(int64_t n, const float* pos, const int64_t* ids, float L, float ll,
                  int64_t* labels) {
  if (n < 0 || (n > 0 && (!pos || !ids || !labels))) return -1;
  if (!(ll > 0.f) || !(L > 0.f)) return -1;
  const float hL = 0.5f * L, ll2 = ll * ll;
  int64_t nc = int64_t(std::floor(double(L) / (1.01 * double(ll))));
  nc = std::max<int64_t>(1, std::min<int64_t>(nc, 1 << 20));
  auto cell_of = [&](int64_t i, int d) {
    int64_t c = int64_t(std::floor(double(pos[3 * i + d]) * double(nc) / double(L)));
    return std::min<int64_t>(std::max<int64_t>(c, 0), nc - 1);
  };
  auto key = [&](int64_t cx, int64_t cy, int64_t cz) { return (cz * nc + cy) * nc + cx; };
  std::vector<std::pair<int64_t, int64_t>> kp(n);
  for (int64_t i = 0; i < n; ++i) kp[i] = {key(cell_of(i, 0), cell_of(i, 1), cell_of(i, 2)), i};
  std::sort(kp.begin(), kp.end());
  std::unordered_map<int64_t, std::pair<int64_t, int64_t>> cells;
  cells.reserve(size_t(n) * 2 + 1);
  for (int64_t s = 0; s < n;) {
    int64_t e = s;
    while (e < n && kp[e].first == kp[s].first) ++e;
    cells[kp[s].first] = {s, e};
    s = e;
  }
  UnionFind uf(n);
  for (const auto& cell : cells) {
    const int64_t k = cell.first;
    const int64_t cx = k % nc, cy = (k / nc) % nc, cz = k / (nc * nc);
    for (int64_t oz = -1; oz <= 1; ++oz)
      for (int64_t oy = -1; oy <= 1; ++oy)
        for (int64_t ox = -1; ox <= 1; ++ox) {
          const int64_t k2 = key((cx + ox + nc) % nc, (cy + oy + nc) % nc, (cz + oz + nc) % nc);
          if (k2 < k) continue;  // each unordered cell pair once (duplicates are harmless)
          auto it = cells.find(k2);
          if (it == cells.end()) continue;
          for (int64_t a = cell.second.first; a < cell.second.second; ++a)
            for (int64_t b = it->second.first; b < it->second.second; ++b) {
              const int64_t i = kp[a].second, j = kp[b].second;
              if (i != j && fof_linked(pos, i, j, L, hL, ll2)) uf.unite(i, j);
            }
        }
  }
  labels_from_uf(n, ids, uf, labels);
  return 0;
}

// CRO sum of a float64 array.
double or_cro_sum(const double* a, int64_t m) {
  return cro_sum(m, [&](int64_t i) { return a[i]; });
}

// One level of 6D FoF on a single node given as float32 u[g][3], v[g][3] (members in ascending
// id order, u already relative to the reference member). Outputs: inv_sx2, inv_sv2, l2 (3
// floats), nn2[g], comp[g] (smallest member position of each member's component).
int or_split_node(int64_t g, const float* u, const float* v, int32_t f_num, int32_t f_den,
                  float* scal_out, float* nn2_out, int64_t* comp_out) {
  return or_split_node_ex(g, u, v, f_num, f_den, -1, 1, scal_out, nn2_out, comp_out);
}

// or_split_node with the search chosen explicitly (pruned: 0 all pairs, 1 k-d tree, -1 by
// size) and the member loops of the k-d tree search spread over `threads`.
int or_split_node_ex(int64_t g, const float* u, const float* v, int32_t f_num, int32_t f_den,
                     int32_t pruned, int32_t threads, float* scal_out, float* nn2_out,
                     int64_t* comp_out) {
  if (g < 2 || f_num <= 0 || f_den <= 0 || f_num > f_den) return -1;
  SplitResult sr;
  split_node(u, v, g, f_num, f_den, sr, std::max(1, int(threads)), pruned);
  scal_out[0] = sr.inv_sx2;
  scal_out[1] = sr.inv_sv2;
  scal_out[2] = sr.l2;
  std::memcpy(nn2_out, sr.nn2.data(), sizeof(float) * g);
  std::memcpy(comp_out, sr.comp.data(), sizeof(int64_t) * g);
  return 0;
}

// Build the hierarchy; returns an opaque handle (free with or_hierarchy_free).
void* or_hierarchy(int64_t n, const float* pos, const float* vel, const int64_t* ids,
                   const int64_t* fof_label, float L, int32_t f_num, int32_t f_den,
                   int32_t min_size, int32_t threads, int64_t* n_nodes, int64_t* n_members) {
  if (n < 0 || f_num <= 0 || f_den <= 0 || f_num > f_den || min_size < 2) return nullptr;
  Hierarchy* h = build_hierarchy(n, pos, vel, ids, fof_label, L, f_num, f_den, min_size, threads);
  *n_nodes = int64_t(h->nodes.size());
  *n_members = int64_t(h->members.size());
  return h;
}

// Copy the hierarchy out: node arrays [n_nodes], member_off [n_nodes + 1],
// member_idx [n_members], deepest [n].
int or_hierarchy_copy(void* handle, int64_t* parent, int32_t* level, int64_t* min_id,
                      int64_t* size, int64_t* member_off, int64_t* member_idx, int64_t* deepest) {
  auto* h = static_cast<Hierarchy*>(handle);
  if (!h) return -1;
  const int64_t nn = int64_t(h->nodes.size());
  for (int64_t q = 0; q < nn; ++q) {
    parent[q] = h->nodes[q].parent;
    level[q] = h->nodes[q].level;
    min_id[q] = h->nodes[q].min_id;
    size[q] = h->nodes[q].size;
    member_off[q] = h->nodes[q].off;
  }
  member_off[nn] = int64_t(h->members.size());
  std::memcpy(member_idx, h->members.data(), sizeof(int64_t) * h->members.size());
  std::memcpy(deepest, h->deepest.data(), sizeof(int64_t) * h->n);
  return 0;
}

// Seed halos, particle assignment and host relations of a hierarchy (assign_seeds above); the
// hierarchy arrays as or_hierarchy_copy gives them, params = or_hierarchy_params.
int or_assign_seeds(int64_t n, const float* pos, const float* vel, float L, int64_t n_nodes,
                    const int64_t* parent, const int64_t* member_off, const int64_t* member_idx,
                    const int64_t* deepest, const float* params, int32_t threads,
                    int64_t* particle_seed, int64_t* node_host, int64_t* node_count) {
  if (n < 0 || n_nodes < 0) return -1;
  return assign_seeds(n, pos, vel, L, n_nodes, parent, member_off, member_idx, deepest, params,
                      std::max(1, int(threads)), particle_seed, node_host, node_count);
}

// Temporal tracking of seed halos between two snapshots of the same particles (matched by id;
// the paper's Summary names temporal tracking, the method is a stated reading): the progenitor
// of a seed h2 of the later snapshot is the seed h1 of the earlier one holding the most of h2's
// particles (ties: the smaller index; -1 when none of h2's particles is in a seed of the earlier
// snapshot); the descendant of h1 is the seed h2 receiving the most of h1's particles (ties:
// the smaller index). Shared counts are returned beside them. Particles absent from one snapshot
// or in no seed are ignored. seed1 / seed2: per particle, a node index or -1 (as or_assign_seeds
// gives them); nn1 / nn2: node counts (outputs are per node, -1 / 0 for nodes that are no seed).
int or_track(int64_t n1, const int64_t* ids1, const int64_t* seed1, int64_t nn1, int64_t n2,
             const int64_t* ids2, const int64_t* seed2, int64_t nn2, int64_t* prog,
             int64_t* prog_shared, int64_t* desc, int64_t* desc_shared) {
  if (n1 < 0 || n2 < 0 || nn1 < 0 || nn2 < 0) return -1;
  std::unordered_map<int64_t, int64_t> where;
  where.reserve(size_t(n1) * 2 + 1);
  for (int64_t i = 0; i < n1; ++i) where[ids1[i]] = seed1[i];
  std::map<std::pair<int64_t, int64_t>, int64_t> shared;  // (h2, h1) -> particles
  for (int64_t j = 0; j < n2; ++j) {
    if (seed2[j] < 0) continue;
    auto it = where.find(ids2[j]);
    if (it == where.end() || it->second < 0) continue;
    shared[{seed2[j], it->second}]++;
  }
  for (int64_t q = 0; q < nn2; ++q) {
    prog[q] = -1;
    prog_shared[q] = 0;
  }
  for (int64_t q = 0; q < nn1; ++q) {
    desc[q] = -1;
    desc_shared[q] = 0;
  }
  for (const auto& kv : shared) {  // ascending (h2, h1): the first maximum has the smaller h1
    const int64_t h2 = kv.first.first, h1 = kv.first.second, c = kv.second;
    if (c > prog_shared[h2]) {
      prog_shared[h2] = c;
      prog[h2] = h1;
    }
  }
  for (const auto& kv : shared) {
    const int64_t h2 = kv.first.first, h1 = kv.first.second, c = kv.second;
    if (c > desc_shared[h1] || (c == desc_shared[h1] && h2 < desc[h1])) {
      desc_shared[h1] = c;
      desc[h1] = h2;
    }
  }
  return 0;
}

// Split parameters of every node: inv_sx2, inv_sv2, l2 (float32 [n_nodes][3]).
int or_hierarchy_params(void* handle, float* params) {
  auto* h = static_cast<Hierarchy*>(handle);
  if (!h) return -1;
  for (size_t q = 0; q < h->nodes.size(); ++q)
    for (int k = 0; k < 3; ++k) params[3 * q + k] = h->nodes[q].scal[k];
  return 0;
}

void or_hierarchy_free(void* handle) { delete static_cast<Hierarchy*>(handle); }

// Unbinding over every node of the hierarchy (member CSR: member_off [n_nodes+1], member_idx).
// Per node with reference member r (its first = smallest-id member) and u = wrap(x - x_r):
//   phi_i  = -(G m) * CRO_j( j == i ? 0 : 1 / sqrt(((Dx*Dx + Dy*Dy) + Dz*Dz) + eps^2) ),
//            D = (double)u_j - (double)u_i, eps^2 = (double)eps * (double)eps;
//   v_bulk = CRO(v) / g;  KE_i = 0.5 * ((dvx*dvx + dvy*dvy) + dvz*dvz), dv = (double)v_i - v_bulk;
//   bound_i = (KE_i + phi_i < 0); N_b = #bound; halo iff N_b >= min_size and
//   bf_den * N_b >= bf_num * g; M_b = N_b * m.
// Outputs per member (CSR order): phi [n_members] (may be NULL), bound [n_members];
// per node: n_bound, is_halo, m_bound.
int or_unbind(int64_t n_nodes, const int64_t* member_off, const int64_t* member_idx,
              const float* pos, const float* vel, float L, float eps, double G, double m,
              int32_t min_size, int32_t bf_num, int32_t bf_den, int32_t threads, double* phi,
              uint8_t* bound, int64_t* n_bound, uint8_t* is_halo, double* m_bound) {
  return or_unbind_iter(n_nodes, member_off, member_idx, pos, vel, L, eps, G, m, min_size, bf_num,
                        bf_den, 1, threads, phi, bound, n_bound, is_halo, m_bound);
}

// or_unbind with iterative passes: pass 1 as above; pass p > 1 recomputes the bulk velocity
// (CRO over the members still bound, the others contributing 0.0, divided by their count) and
// the potential of every member still bound over the members still bound (the others
// contributing 0.0 like the self term), re-flags them, and leaves the others unbound; it stops
// after `passes` passes or when a pass changes no flag. phi holds each member's potential from
// the last pass that evaluated it.
int or_unbind_iter(int64_t n_nodes, const int64_t* member_off, const int64_t* member_idx,
                   const float* pos, const float* vel, float L, float eps, double G, double m,
                   int32_t min_size, int32_t bf_num, int32_t bf_den, int32_t passes,
                   int32_t threads, double* phi, uint8_t* bound, int64_t* n_bound,
                   uint8_t* is_halo, double* m_bound) {
  if (n_nodes < 0 || bf_den <= 0 || passes < 1) return -1;
  const double Gm = G * m;
  const double eps2 = double(eps) * double(eps);
  parallel_for(n_nodes, threads, [&](int64_t q) {
    const int64_t off = member_off[q], g = member_off[q + 1] - member_off[q];
    const int64_t* mem = member_idx + off;
    std::vector<float> u;
    unwrap_node(pos, mem, g, L, u);
    std::vector<uint8_t> in(g, 1), next(g, 0);
    int64_t nb = 0;
    for (int32_t pass = 0; pass < passes; ++pass) {
      int64_t cnt = 0;
      for (int64_t a = 0; a < g; ++a) cnt += in[a];
      if (cnt == 0) break;
      double vb[3];
      for (int d = 0; d < 3; ++d)
        vb[d] = cro_sum(g, [&](int64_t a) { return in[a] ? double(vel[3 * mem[a] + d]) : 0.0; }) / double(cnt);
      nb = 0;
      bool changed = false;
      for (int64_t i = 0; i < g; ++i) {
        next[i] = 0;
        if (!in[i]) continue;
        double p;
        const bool b = member_energy(u.data(), vel, mem, g, i, vb, eps2, Gm, &p, in.data());
        if (phi) phi[off + i] = p;
        next[i] = b ? 1 : 0;
        nb += b ? 1 : 0;
        changed = changed || !b;
      }
      in.swap(next);
      if (!changed) break;
    }
    for (int64_t i = 0; i < g; ++i) bound[off + i] = in[i];
    n_bound[q] = nb;
    is_halo[q] = (nb >= min_size && int64_t(bf_den) * nb >= int64_t(bf_num) * g) ? 1 : 0;
    m_bound[q] = double(nb) * m;
  });
  return 0;
}

// Unbinding of selected members of ONE node (mem: its g particle indices, ascending id), by the
// definition of or_unbind: the node's bulk velocity from all its members, then phi_i, KE_i and
// the flag of each member sample[s] (positions in mem), the samples spread over threads.
int or_unbind_sample(int64_t g, const int64_t* mem, const float* pos, const float* vel, float L,
                     float eps, double G, double m, int64_t k, const int64_t* sample,
                     int32_t threads, double* phi_out, uint8_t* bound_out) {
  if (g < 1 || k < 0) return -1;
  for (int64_t s = 0; s < k; ++s)
    if (sample[s] < 0 || sample[s] >= g) return -1;
  const double Gm = G * m;
  const double eps2 = double(eps) * double(eps);
  std::vector<float> u;
  unwrap_node(pos, mem, g, L, u);
  double vb[3];
  bulk_velocity(vel, mem, g, vb);
  parallel_for(k, threads, [&](int64_t s) {
    double p;
    bound_out[s] = member_energy(u.data(), vel, mem, g, sample[s], vb, eps2, Gm, &p) ? 1 : 0;
    phi_out[s] = p;
  });
  return 0;
}

// Halo properties per node over its bound members (CRO sums over all members in ascending id
// order, unbound members contributing 0.0), 20 float64 per node:
//   [0] n, [1] n_bound, [2] is_halo, [3] m_bound, [4..6] centre, [7..9] bulk velocity,
//   [10] sigma_x, [11] sigma_v, [12] r_vir, [13..18] inertia xx yy zz xy xz yz, [19] unused 0.
// centre = x_r + mean(u) wrapped once into [0, L); sigma^2 = sum_d (CRO(w_d^2)/N_b - mean_d^2)
// (clamped at 0); r_vir = cbrt(3 M_b / (4 pi 200 rho_bar)), rho_bar = n_total m / L^3;
// inertia I_ab = CRO((u_a - mean_a)(u_b - mean_b)) / N_b. All zero except [0..3] when N_b = 0.
int or_props(int64_t n_nodes, const int64_t* member_off, const int64_t* member_idx,
             const float* pos, const float* vel, const uint8_t* bound, const uint8_t* is_halo,
             float L, double m, int64_t n_total, int32_t threads, double* props) {
  if (n_nodes < 0 || n_total <= 0) return -1;
  const double rho_bar = double(n_total) * m / (double(L) * double(L) * double(L));
  const double pi = 3.14159265358979323846;
  parallel_for(n_nodes, threads, [&](int64_t q) {
    const int64_t off = member_off[q], g = member_off[q + 1] - member_off[q];
    const int64_t* mem = member_idx + off;
    const uint8_t* bd = bound + off;
    double* P = props + 20 * q;
    for (int k = 0; k < 20; ++k) P[k] = 0.0;
    std::vector<float> u;
    unwrap_node(pos, mem, g, L, u);
    int64_t nb = 0;
    for (int64_t a = 0; a < g; ++a) nb += bd[a] ? 1 : 0;
    P[0] = double(g);
    P[1] = double(nb);
    P[2] = is_halo[q] ? 1.0 : 0.0;
    P[3] = double(nb) * m;
    if (nb == 0) return;
    const double nbd = double(nb);
    double mu[3], mv[3];
    double varx = 0.0, varv = 0.0;
    for (int d = 0; d < 3; ++d) {
      mu[d] = cro_sum(g, [&](int64_t a) { return bd[a] ? double(u[3 * a + d]) : 0.0; }) / nbd;
      mv[d] = cro_sum(g, [&](int64_t a) { return bd[a] ? double(vel[3 * mem[a] + d]) : 0.0; }) / nbd;
      const double qx = cro_sum(g, [&](int64_t a) {
        return bd[a] ? double(u[3 * a + d]) * double(u[3 * a + d]) : 0.0; });
      const double qv = cro_sum(g, [&](int64_t a) {
        return bd[a] ? double(vel[3 * mem[a] + d]) * double(vel[3 * mem[a] + d]) : 0.0; });
      const double tx = qx / nbd - mu[d] * mu[d];
      const double tv = qv / nbd - mv[d] * mv[d];
      varx = (d == 0) ? tx : varx + tx;
      varv = (d == 0) ? tv : varv + tv;
    }
    for (int d = 0; d < 3; ++d) {
      double c = double(pos[3 * mem[0] + d]) + mu[d];
      if (c < 0.0) c = c + double(L);
      else if (c >= double(L)) c = c - double(L);
      P[4 + d] = c;
      P[7 + d] = mv[d];
    }
    P[10] = std::sqrt(varx > 0.0 ? varx : 0.0);
    P[11] = std::sqrt(varv > 0.0 ? varv : 0.0);
    P[12] = std::cbrt(3.0 * P[3] / (4.0 * pi * 200.0 * rho_bar));
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
      P[13 + k] = cro_sum(g, [&](int64_t a) {
        if (!bd[a]) return 0.0;
        const double da = double(u[3 * a + ia[k]]) - mu[ia[k]];
        const double db = double(u[3 * a + ib[k]]) - mu[ib[k]];
        return da * db;
      }) / nbd;
    }
  });
  return 0;
}

}  // extern "C"

// =============================================================================================
// Surrogate MLP oracle: float64 forward and gradient of the 8 -> 64 -> 64 -> 1 ReLU network on
// the same parameter vector layout as the device (W1 [8][64] at 0, b1 at 512, W2 [64][64] at
// 576, b2 at 4672, W3 [64] at 4736, b3 at 4800). With round != 0, inputs, weights, hidden
// activations and the hidden-layer error signals are rounded to bf16 (round to nearest even,
// via float32) at the points where the device rounds them; sums are float64. With round == 0
// everything is float64 (the form a finite-difference check can verify).
namespace {

inline double bf16r(double v) {
  float f = float(v);
  uint32_t b;
  std::memcpy(&b, &f, 4);
  const uint32_t lsb = (b >> 16) & 1u;
  b = (b + 0x7fffu + lsb) & 0xffff0000u;
  float r;
  std::memcpy(&r, &b, 4);
  return double(r);
}

struct MlpFwd {
  double x[8], h1[64], h2[64], y;
};

void mlp_fwd1(const float* xin, const float* P, bool rnd, MlpFwd& f) {
  auto R = [&](double v) { return rnd ? bf16r(v) : v; };
  for (int i = 0; i < 8; ++i) f.x[i] = R(xin[i]);
  for (int o = 0; o < 64; ++o) {
    double z = P[512 + o];
    for (int i = 0; i < 8; ++i) z += R(P[i * 64 + o]) * f.x[i];
    f.h1[o] = R(z > 0.0 ? z : 0.0);
  }
  for (int o = 0; o < 64; ++o) {
    double z = P[4672 + o];
    for (int i = 0; i < 64; ++i) z += R(P[576 + i * 64 + o]) * f.h1[i];
    f.h2[o] = R(z > 0.0 ? z : 0.0);
  }
  double y = P[4800];
  for (int k = 0; k < 64; ++k) y += R(P[4736 + k]) * f.h2[k];
  f.y = y;
}

}  // namespace

extern "C" {

int or_mlp_forward(int64_t n, const float* x, const float* params, int32_t round, double* y) {
  if (n < 0) return -1;
  for (int64_t s = 0; s < n; ++s) {
    MlpFwd f;
    mlp_fwd1(x + 8 * s, params, round != 0, f);
    y[s] = f.y;
  }
  return 0;
}

// Gradient of L = (1/n) sum (y - t)^2 with respect to the parameter vector; also returns the
// sum of squared errors.
int or_mlp_gradient(int64_t n, const float* x, const float* t, const float* params, int32_t round,
                    double* grad, double* sse) {
  if (n <= 0) return -1;
  const bool rnd = round != 0;
  auto R = [&](double v) { return rnd ? bf16r(v) : v; };
  for (int p = 0; p < 4801; ++p) grad[p] = 0.0;
  double tot = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    MlpFwd f;
    mlp_fwd1(x + 8 * s, params, rnd, f);
    const double e = f.y - double(t[s]);
    tot += e * e;
    const double dy = rnd ? double(float(2.0 * double(float(f.y) - t[s]) / double(n))) : 2.0 * e / double(n);
    grad[4800] += dy;
    double dz2[64], dz1[64];
    for (int k = 0; k < 64; ++k) {
      grad[4736 + k] += dy * f.h2[k];
      dz2[k] = R(f.h2[k] > 0.0 ? dy * R(params[4736 + k]) : 0.0);
      grad[4672 + k] += dz2[k];
    }
    for (int i = 0; i < 64; ++i) {
      double dh = 0.0;
      for (int o = 0; o < 64; ++o) {
        grad[576 + i * 64 + o] += f.h1[i] * dz2[o];
        dh += R(params[576 + i * 64 + o]) * dz2[o];
      }
      dz1[i] = R(f.h1[i] > 0.0 ? dh : 0.0);
      grad[512 + i] += dz1[i];
    }
    for (int i = 0; i < 8; ++i)
      for (int o = 0; o < 64; ++o) grad[i * 64 + o] += f.x[i] * dz1[o];
  }
  if (sse) *sse = tot;
  return 0;
}

}  // extern "C"
