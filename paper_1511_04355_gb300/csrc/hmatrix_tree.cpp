// Cluster tree and block partition of the H-matrix far field (host, IEEE double, no
// floating-point contraction: see hmatrix_host.h).  Hierarchical matrices: Hackbusch 1999,
// "A sparse matrix arithmetic based on H-matrices"; the standard admissibility condition
// max(diam s, diam t) <= eta dist(s, t) on axis-parallel bounding boxes.
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "hmatrix_host.h"

namespace bem {
namespace hm {

namespace {

struct Builder {
  const double* c;     // centroids, 3 per element
  const double* vlo;   // per element vertex bounds
  const double* vhi;
  int leaf;
  Tree* t;

  int32_t build(int32_t b, int32_t n) {
    const int32_t id = (int32_t)t->begin.size();
    t->begin.push_back(b);
    t->size.push_back(n);
    t->left.push_back(-1);
    t->right.push_back(-1);
    double lo[3], hi[3], cmin[3], cmax[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = cmin[k] = INFINITY;
      hi[k] = cmax[k] = -INFINITY;
    }
    int32_t* idx = t->perm.data() + b;
    for (int32_t a = 0; a < n; ++a) {
      const int32_t e = idx[a];
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], vlo[3 * e + k]);
        hi[k] = std::max(hi[k], vhi[3 * e + k]);
        cmin[k] = std::min(cmin[k], c[3 * e + k]);
        cmax[k] = std::max(cmax[k], c[3 * e + k]);
      }
    }
    for (int k = 0; k < 3; ++k) {
      t->lo.push_back(lo[k]);
      t->hi.push_back(hi[k]);
    }
    if (n <= leaf) return id;
    int ax = 0;
    double best = cmax[0] - cmin[0];
    for (int k = 1; k < 3; ++k) {
      const double ext = cmax[k] - cmin[k];
      if (ext > best) {
        best = ext;
        ax = k;
      }
    }
    const double* cc = c;
    std::sort(idx, idx + n, [cc, ax](int32_t p, int32_t q) {
      const double a = cc[3 * p + ax], b2 = cc[3 * q + ax];
      return a < b2 || (a == b2 && p < q);
    });
    const int32_t h = n / 2;
    const int32_t l = build(b, h);
    const int32_t r = build(b + h, n - h);
    t->left[id] = l;
    t->right[id] = r;
    return id;
  }
};

double box_distance(const Tree& t, int32_t a, int32_t b) {
  double g[3];
  for (int k = 0; k < 3; ++k)
    g[k] = std::max(0.0, std::max(t.lo[3 * b + k] - t.hi[3 * a + k], t.lo[3 * a + k] - t.hi[3 * b + k]));
  const double s = g[0] * g[0] + g[1] * g[1];
  return std::sqrt(s + g[2] * g[2]);
}

struct Splitter {
  const Tree& t;
  double eta;
  int max_block;
  Partition& p;
  void rec(int32_t a, int32_t b) {
    if (t.size[a] <= max_block && t.size[b] <= max_block) {
      const double d = box_distance(t, a, b);
      if (d > 0.0 && std::max(t.diam[a], t.diam[b]) <= eta * d) {
        p.lowrank.push_back(a);
        p.lowrank.push_back(b);
        return;
      }
    }
    const bool la = t.leaf(a), lb = t.leaf(b);
    if (la && lb) {
      p.dense.push_back(a);
      p.dense.push_back(b);
      return;
    }
    const int32_t ta[2] = {la ? a : t.left[a], la ? -1 : t.right[a]};
    const int32_t tb[2] = {lb ? b : t.left[b], lb ? -1 : t.right[b]};
    for (int x = 0; x < 2; ++x) {
      if (ta[x] < 0) continue;
      for (int y = 0; y < 2; ++y) {
        if (tb[y] < 0) continue;
        rec(ta[x], tb[y]);
      }
    }
  }
};

}  // namespace

void cluster_tree(const double* verts, int64_t nv, const int32_t* tris, int64_t ne, int leaf, Tree& t) {
  if (ne <= 0 || nv <= 0 || leaf < 1) throw std::invalid_argument("cluster tree: empty mesh or leaf < 1");
  std::vector<double> c(3 * ne), vlo(3 * ne), vhi(3 * ne);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* v = tris + 3 * e;
    for (int j = 0; j < 3; ++j)
      if (v[j] < 0 || v[j] >= nv) throw std::invalid_argument("cluster tree: vertex index out of range");
    for (int k = 0; k < 3; ++k) {
      const double p0 = verts[3 * v[0] + k], p1 = verts[3 * v[1] + k], p2 = verts[3 * v[2] + k];
      c[3 * e + k] = ((p0 + p1) + p2) / 3.0;
      vlo[3 * e + k] = std::min(std::min(p0, p1), p2);
      vhi[3 * e + k] = std::max(std::max(p0, p1), p2);
    }
  }
  t = Tree();
  t.perm.resize(ne);
  for (int64_t e = 0; e < ne; ++e) t.perm[e] = (int32_t)e;
  Builder bld{c.data(), vlo.data(), vhi.data(), leaf, &t};
  bld.build(0, (int32_t)ne);
  const int64_t n = t.n();
  t.diam.resize(n);
  for (int64_t k = 0; k < n; ++k) {
    const double d0 = t.hi[3 * k] - t.lo[3 * k], d1 = t.hi[3 * k + 1] - t.lo[3 * k + 1],
                 d2 = t.hi[3 * k + 2] - t.lo[3 * k + 2];
    const double s = d0 * d0 + d1 * d1;
    t.diam[k] = std::sqrt(s + d2 * d2);
  }
}

void block_partition(const Tree& t, double eta, int max_block, Partition& p) {
  p = Partition();
  Splitter sp{t, eta, max_block, p};
  sp.rec(0, 0);
}

}  // namespace hm
}  // namespace bem
