// Host-side scene build: input validation, a binned-SAH binary BVH refined by
// subtree reinsertion and laid out for the GPU traversal (binary, 4-wide and
// 8-wide nodes), triangles in leaf order, and the per-segment area tables
// used for light selection.  Compiled without floating-point
// contraction so the FP64 area sums are reproducible across hosts.
#include <algorithm>
#include <functional>
#include <cmath>
#include <queue>
#include <cstring>
#include <string>
#include <vector>

#include "ipt_internal.h"

namespace ipt {
namespace {

struct Box {
  double lo[3], hi[3];
  void reset() {
    for (int k = 0; k < 3; ++k) {
      lo[k] = 1e300;
      hi[k] = -1e300;
    }
  }
  void grow(const double* p) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], p[k]);
      hi[k] = std::max(hi[k], p[k]);
    }
  }
  void grow(const Box& b) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], b.lo[k]);
      hi[k] = std::max(hi[k], b.hi[k]);
    }
  }
  double area() const {
    const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    if (dx < 0 || dy < 0 || dz < 0) return 0.0;
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  }
};

struct BNode {
  Box box;
  int left = -1, right = -1;
  uint32_t first = 0, count = 0;
  int depth = 0;
};

constexpr int kBins = 32;
constexpr double kCtrav = 1.0;  // SAH: cost of a node step relative to a triangle test
constexpr uint32_t kMaxLeaf = 8;
constexpr int kMedianDepth = 48;

struct Builder {
  std::vector<Box> pbox;
  std::vector<double> cen;  // 3 per primitive
  std::vector<uint32_t> order;
  std::vector<BNode> nodes;

  int make_node(uint32_t b, uint32_t e, int depth) {
    BNode n;
    n.box.reset();
    for (uint32_t i = b; i < e; ++i) n.box.grow(pbox[order[i]]);
    n.first = b;
    n.count = e - b;
    n.depth = depth;
    nodes.push_back(n);
    return (int)nodes.size() - 1;
  }

  // Returns split position in [b, e] or b when the range should stay a leaf.
  uint32_t split(uint32_t b, uint32_t e, int depth, bool force) {
    const uint32_t n = e - b;
    Box cb;
    cb.reset();
    for (uint32_t i = b; i < e; ++i) cb.grow(&cen[3 * order[i]]);
    int axis = 0;
    double ext[3];
    for (int k = 0; k < 3; ++k) ext[k] = cb.hi[k] - cb.lo[k];
    axis = (ext[0] >= ext[1] && ext[0] >= ext[2]) ? 0 : (ext[1] >= ext[2] ? 1 : 2);
    auto median = [&](int ax) {
      const uint32_t mid = b + n / 2;
      std::nth_element(order.begin() + b, order.begin() + mid, order.begin() + e, [&](uint32_t x, uint32_t y) {
        const double cx = cen[3 * x + ax], cy = cen[3 * y + ax];
        return cx < cy || (cx == cy && x < y);
      });
      return mid;
    };
    if (ext[axis] <= 0.0) {
      if (n <= kMaxLeaf && !force) return b;
      return median(axis);
    }
    if (depth >= kMedianDepth) {
      if (n <= 2 && !force) return b;
      return median(axis);
    }
    Box parent;
    parent.reset();
    for (uint32_t i = b; i < e; ++i) parent.grow(pbox[order[i]]);
    const double pa = parent.area();
    double best = 1e300;
    int best_axis = -1, best_bin = -1;
    for (int ax = 0; ax < 3; ++ax) {
      if (ext[ax] <= 0.0) continue;
      Box bins[kBins];
      uint32_t cnt[kBins] = {0};
      for (int k = 0; k < kBins; ++k) bins[k].reset();
      const double scale = kBins / ext[ax];
      for (uint32_t i = b; i < e; ++i) {
        int k = (int)((cen[3 * order[i] + ax] - cb.lo[ax]) * scale);
        k = std::min(std::max(k, 0), kBins - 1);
        cnt[k]++;
        bins[k].grow(pbox[order[i]]);
      }
      double right_area[kBins];
      uint32_t right_cnt[kBins];
      Box acc;
      acc.reset();
      uint32_t c = 0;
      for (int k = kBins - 1; k >= 1; --k) {
        acc.grow(bins[k]);
        c += cnt[k];
        right_area[k] = acc.area();
        right_cnt[k] = c;
      }
      acc.reset();
      c = 0;
      for (int k = 0; k < kBins - 1; ++k) {
        acc.grow(bins[k]);
        c += cnt[k];
        if (c == 0 || right_cnt[k + 1] == 0) continue;
        const double cost = kCtrav + (acc.area() * c + right_area[k + 1] * right_cnt[k + 1]) / pa;
        if (cost < best) {
          best = cost;
          best_axis = ax;
          best_bin = k;
        }
      }
    }
    if (best_axis < 0) return median(axis);
    if (!force && n <= kMaxLeaf && best >= (double)n) return b;
    const double scale = kBins / ext[best_axis];
    auto it = std::partition(order.begin() + b, order.begin() + e, [&](uint32_t x) {
      int k = (int)((cen[3 * x + best_axis] - cb.lo[best_axis]) * scale);
      k = std::min(std::max(k, 0), kBins - 1);
      return k <= best_bin;
    });
    uint32_t mid = (uint32_t)(it - order.begin());
    if (mid == b || mid == e) mid = median(best_axis);
    return mid;
  }

  void build(uint32_t n) {
    order.resize(n);
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    nodes.reserve(2 * (size_t)n + 2);
    make_node(0, n, 0);
    std::vector<int> work = {0};
    while (!work.empty()) {
      const int ni = work.back();
      work.pop_back();
      const uint32_t b = nodes[ni].first, e = b + nodes[ni].count;
      const int depth = nodes[ni].depth;
      const bool force = (ni == 0 && e - b >= 2) || (e - b > kMaxLeaf);
      const uint32_t mid = (e - b >= 2) ? split(b, e, depth, force) : b;
      if (mid == b || mid == e) continue;  // leaf
      const int l = make_node(b, mid, depth + 1);
      const int r = make_node(mid, e, depth + 1);
      nodes[ni].left = l;
      nodes[ni].right = r;
      work.push_back(r);
      work.push_back(l);
    }
  }
};

// Insertion-based optimisation of the binary tree (after Bittner, Hapala
// and Havran, "Fast insertion-based optimization of bounding volume
// hierarchies", 2013): each subtree in turn is taken out and put back as the
// sibling of the node where the tree's surface-area cost grows least (a
// best-first search over the induced cost of the ancestors).  Leaves keep
// their triangle ranges; the root stays node 0.
struct Reinserter {
  std::vector<BNode>& nd;
  std::vector<int> parent;

  explicit Reinserter(std::vector<BNode>& n) : nd(n), parent(n.size(), -1) {
    for (size_t i = 0; i < nd.size(); ++i)
      if (nd[i].left >= 0) {
        parent[nd[i].left] = (int)i;
        parent[nd[i].right] = (int)i;
      }
  }
  static double merged_area(const Box& a, const Box& b) {
    Box r = a;
    r.grow(b);
    return r.area();
  }
  void refit(int i) {
    for (; i >= 0; i = parent[i]) {
      nd[i].box = nd[nd[i].left].box;
      nd[i].box.grow(nd[nd[i].right].box);
    }
  }
  // takes subtree x out (its parent is bypassed); returns the freed parent
  int take_out(int x) {
    const int p = parent[x], g = parent[p];
    const int sib = nd[p].left == x ? nd[p].right : nd[p].left;
    (nd[g].left == p ? nd[g].left : nd[g].right) = sib;
    parent[sib] = g;
    refit(g);
    return p;
  }
  // the node whose new parent (shared with a subtree of box b) adds least cost
  int best_sibling(const Box& b) const {
    struct Cand {
      double induced;
      int n;
      bool operator<(const Cand& o) const { return induced > o.induced; }
    };
    const double ab = b.area();
    int best = 0;
    double best_cost = merged_area(nd[0].box, b);
    std::priority_queue<Cand> q;
    q.push({0.0, 0});
    while (!q.empty()) {
      const Cand c = q.top();
      q.pop();
      if (c.induced + ab >= best_cost) break;
      const double total = c.induced + merged_area(nd[c.n].box, b);
      if (total < best_cost) {
        best_cost = total;
        best = c.n;
      }
      if (nd[c.n].left >= 0) {
        const double induced = total - nd[c.n].box.area();
        if (induced + ab < best_cost) {
          q.push({induced, nd[c.n].left});
          q.push({induced, nd[c.n].right});
        }
      }
    }
    return best;
  }
  // puts subtree x back as the sibling of node `at`, under the freed node p
  void put_back(int x, int p, int at) {
    const int g = parent[at];
    nd[p].left = at;
    nd[p].right = x;
    parent[at] = p;
    parent[x] = p;
    parent[p] = g;
    if (g >= 0) {
      (nd[g].left == at ? nd[g].left : nd[g].right) = p;
      refit(p);
      return;
    }
    // `at` is the root: the new parent takes index 0, the old root index p
    std::swap(nd[0], nd[p]);
    nd[0].left = p;
    for (int c : {nd[p].left, nd[p].right})
      if (c >= 0) parent[c] = p;
    parent[p] = 0;
    parent[x] = 0;
    parent[0] = -1;
    refit(0);
  }
  void run(int passes) {
    for (int it = 0; it < passes; ++it)
      for (int x = 1; x < (int)nd.size(); ++x) {
        const int p = parent[x];
        if (p <= 0) continue;  // the root's children stay
        const int freed = take_out(x);
        put_back(x, freed, best_sibling(nd[x].box));
      }
  }
};

// Renumbers the tree in pre-order from the root (parents before children,
// as the collapse to wide nodes expects) and sets every node's depth.
void preorder(std::vector<BNode>& nd) {
  std::vector<BNode> out;
  out.reserve(nd.size());
  std::vector<std::pair<int, int>> st = {{0, -1}};  // (old index, new parent index)
  while (!st.empty()) {
    const auto [o, np] = st.back();
    st.pop_back();
    BNode n = nd[o];
    n.depth = np < 0 ? 0 : out[np].depth + 1;
    const int me = (int)out.size();
    if (np >= 0) (out[np].left == -2 ? out[np].left : out[np].right) = me;
    const int l = n.left, r = n.right;
    if (l >= 0) {
      n.left = -2;  // filled in when the children are emitted
      n.right = -2;
    }
    out.push_back(n);
    if (l >= 0) {
      st.push_back({r, me});
      st.push_back({l, me});
    }
  }
  nd.swap(out);
}

// 4-wide node with 8-bit child boxes (64 bytes, 16 words):
//   w0..w2: origin p (float bits); w3, w14, w15: 2^15 * scale of the x, y
//   and z axes (float bits); w4..w7: child links (inner node index, or a
//   leaf code as in the binary layout); w8: lo.x of children 0..3 (one byte
//   each), w9: hi.x, w10: lo.y, w11: hi.y, w12: lo.z, w13: hi.z.  A child
//   box is p + q * scale per axis, the scale the smallest float for which 255
//   codes span the node's box (at most one code of slack per side).
// 8-wide node (96 bytes, 24 words): w0..w2 origin, w3 exponents | mask of
//   occupied slots << 24; per axis k, w4+4k..w5+4k the lower bytes and
//   w6+4k..w7+4k the upper bytes of slots 0..3 and 4..7; w16..w23 the
//   slots' links (the first 64 bytes are all a node test reads).
// An 8-wide child box is p + q * 2^(e - 127) per axis, rounded outward so
// that it contains the child's (padded) box in float arithmetic.
struct Quantizer {
  float p;
  int e;  // biased exponent of the scale
  float scale() const {
    uint32_t bits = (uint32_t)e << 23;
    float f;
    std::memcpy(&f, &bits, 4);
    return f;
  }
};

Quantizer make_axis(double lo, double hi) {
  Quantizer q;
  q.p = std::nextafter((float)lo, -INFINITY);
  const double ext = std::max(hi - (double)q.p, 1e-30);
  int e2 = (int)std::ceil(std::log2(ext / 255.0));
  // the largest code (255) must reach past hi
  for (;;) {
    const double s = std::ldexp(1.0, e2);
    if ((double)q.p + 255.0 * s >= hi) break;
    ++e2;
  }
  // coordinates are at most 1e30 in magnitude, so e2 + 127 stays far below
  // 239, the largest exponent traversal accepts (it adds 15 to it)
  q.e = std::min(std::max(e2 + 127, 1), 239);
  return q;
}

uint32_t q_lo(const Quantizer& a, double lo) {
  const float s = a.scale();
  int q = (int)std::floor((lo - (double)a.p) / (double)s);
  q = std::min(std::max(q, 0), 255);
  while (q > 0 && (double)(a.p + (float)q * s) > lo) --q;
  return (uint32_t)q;
}

uint32_t q_hi(const Quantizer& a, double hi) {
  const float s = a.scale();
  int q = (int)std::ceil((hi - (double)a.p) / (double)s);
  q = std::min(std::max(q, 0), 255);
  while (q < 255 && (double)(a.p + (float)q * s) < hi) ++q;
  return (uint32_t)q;
}

// 4-wide nodes: any float scale (the traversal reads it from the node).
struct ScaleQuantizer {
  float p, s;  // plane q of the axis at p + q * s (exact in double)
};

ScaleQuantizer make_scale_axis(double lo, double hi) {
  ScaleQuantizer q;
  q.p = std::nextafter((float)lo, -INFINITY);
  q.s = (float)std::max((hi - (double)q.p) / 255.0, 1e-30);
  while ((double)q.p + 255.0 * (double)q.s < hi) q.s = std::nextafter(q.s, INFINITY);
  return q;
}

uint32_t q_lo(const ScaleQuantizer& a, double lo) {
  int q = (int)std::floor((lo - (double)a.p) / (double)a.s);
  q = std::min(std::max(q, 0), 255);
  while (q > 0 && (double)a.p + q * (double)a.s > lo) --q;
  return (uint32_t)q;
}

uint32_t q_hi(const ScaleQuantizer& a, double hi) {
  int q = (int)std::ceil((hi - (double)a.p) / (double)a.s);
  q = std::min(std::max(q, 0), 255);
  while (q < 255 && (double)a.p + q * (double)a.s < hi) ++q;
  return (uint32_t)q;
}

inline float down(double x) { return std::nextafter((float)x, -INFINITY); }
inline float up(double x) { return std::nextafter((float)x, INFINITY); }
inline float bits_f(uint32_t v) {
  float f;
  std::memcpy(&f, &v, 4);
  return f;
}

}  // namespace

bool build_scene(const float* pos, uint32_t n_vert, const float* nrm, const uint32_t* idx,
                 uint32_t n_tri, const uint32_t* tri_seg, uint32_t n_seg, HostScene* out,
                 std::string* err) {
  if (!pos || !idx || !tri_seg || !out) {
    *err = "null geometry pointer";
    return false;
  }
  if (n_tri == 0 || n_vert == 0 || n_seg == 0) {
    *err = "scene needs at least one vertex, triangle and segment";
    return false;
  }
  if (n_tri >= (1u << 28)) {
    *err = "too many triangles (limit 2^28)";
    return false;
  }
  double maxabs = 0.0;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (uint64_t i = 0; i < 3ull * n_vert; ++i) {
    if (!std::isfinite(pos[i])) {
      *err = "non-finite vertex coordinate at vertex " + std::to_string(i / 3);
      return false;
    }
    maxabs = std::max(maxabs, std::fabs((double)pos[i]));
    if (maxabs > 1e30) {
      // keeps every 4-wide node's scale exponent small enough for traversal
      *err = "vertex coordinate beyond 1e30 at vertex " + std::to_string(i / 3);
      return false;
    }
    lo[i % 3] = std::min(lo[i % 3], (double)pos[i]);
    hi[i % 3] = std::max(hi[i % 3], (double)pos[i]);
  }
  if (nrm)
    for (uint64_t i = 0; i < n_vert; ++i) {
      const double x = nrm[3 * i], y = nrm[3 * i + 1], z = nrm[3 * i + 2];
      if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z) || x * x + y * y + z * z == 0.0) {
        *err = "invalid vertex normal at vertex " + std::to_string(i);
        return false;
      }
    }
  HostScene& s = *out;
  s.n_tri = n_tri;
  s.n_seg = n_seg;
  s.diameter = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                         (hi[2] - lo[2]) * (hi[2] - lo[2]));
  std::vector<double> area(n_tri);
  Builder B;
  B.pbox.resize(n_tri);
  B.cen.resize(3 * (size_t)n_tri);
  for (uint32_t t = 0; t < n_tri; ++t) {
    double p[3][3];
    for (int j = 0; j < 3; ++j) {
      const uint32_t v = idx[3 * t + j];
      if (v >= n_vert) {
        *err = "vertex index out of range in triangle " + std::to_string(t);
        return false;
      }
      for (int k = 0; k < 3; ++k) p[j][k] = pos[3 * v + k];
    }
    if (tri_seg[t] >= n_seg) {
      *err = "segment id out of range in triangle " + std::to_string(t);
      return false;
    }
    const double e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
    const double e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
    const double cx = e1[1] * e2[2] - e1[2] * e2[1];
    const double cy = e1[2] * e2[0] - e1[0] * e2[2];
    const double cz = e1[0] * e2[1] - e1[1] * e2[0];
    const double len = std::sqrt(cx * cx + cy * cy + cz * cz);
    area[t] = 0.5 * len;
    if (!(area[t] > 0.0)) {
      *err = "degenerate (zero-area) triangle " + std::to_string(t);
      return false;
    }
    B.pbox[t].reset();
    for (int j = 0; j < 3; ++j) B.pbox[t].grow(p[j]);
    // binned by the centre of the triangle's box (on the 61k room a 3.4% lower
    // binary SAH cost than binning by the vertex mean)
    for (int k = 0; k < 3; ++k) B.cen[3 * t + k] = 0.5 * (B.pbox[t].lo[k] + B.pbox[t].hi[k]);
  }
  B.build(n_tri);
  {
    // three passes of subtree reinsertion (one above a million triangles);
    // kept unless it deepens the tree beyond what the traversal stack holds
    std::vector<BNode> keep = B.nodes;
    Reinserter(B.nodes).run(n_tri > (1u << 20) ? 1 : 3);
    preorder(B.nodes);
    int deepest = 0;
    for (const BNode& n : B.nodes) deepest = std::max(deepest, n.depth);
    if (deepest > 48) B.nodes.swap(keep);
  }

  // inner nodes in depth-first order; children boxes stored in the parent
  const double pad = maxabs * 1e-6 + 1e-30;
  std::vector<int> gpu_index(B.nodes.size(), -1);
  std::vector<int> inner;
  {
    std::vector<int> st = {0};
    while (!st.empty()) {
      const int n = st.back();
      st.pop_back();
      if (B.nodes[n].left < 0) continue;
      gpu_index[n] = (int)inner.size();
      inner.push_back(n);
      st.push_back(B.nodes[n].right);
      st.push_back(B.nodes[n].left);
    }
  }
  auto leaf_code = [&](const BNode& l) {
    return -(int)((l.first << 3) | (l.count - 1)) - 1;
  };
  uint32_t max_depth = 0;
  for (const BNode& n : B.nodes) max_depth = std::max<uint32_t>(max_depth, (uint32_t)n.depth);
  s.depth = max_depth;
  if (inner.empty()) {
    // single triangle: a root whose second child can never be hit
    s.n_nodes = 1;
    s.nodes.assign(16, 0.0f);
    const Box& b = B.nodes[0].box;
    float* q = s.nodes.data();
    q[0] = down(b.lo[0] - pad); q[1] = up(b.hi[0] + pad); q[2] = down(b.lo[1] - pad); q[3] = up(b.hi[1] + pad);
    q[4] = INFINITY; q[5] = -INFINITY; q[6] = INFINITY; q[7] = -INFINITY;
    q[8] = down(b.lo[2] - pad); q[9] = up(b.hi[2] + pad); q[10] = INFINITY; q[11] = -INFINITY;
    const int code = leaf_code(B.nodes[0]);
    std::memcpy(&q[12], &code, 4);
    std::memcpy(&q[13], &code, 4);
  } else {
    s.n_nodes = (uint32_t)inner.size();
    s.nodes.assign(16 * (size_t)inner.size(), 0.0f);
    for (size_t i = 0; i < inner.size(); ++i) {
      const BNode& n = B.nodes[inner[i]];
      const BNode& a = B.nodes[n.left];
      const BNode& c = B.nodes[n.right];
      float* q = &s.nodes[16 * i];
      q[0] = down(a.box.lo[0] - pad); q[1] = up(a.box.hi[0] + pad);
      q[2] = down(a.box.lo[1] - pad); q[3] = up(a.box.hi[1] + pad);
      q[4] = down(c.box.lo[0] - pad); q[5] = up(c.box.hi[0] + pad);
      q[6] = down(c.box.lo[1] - pad); q[7] = up(c.box.hi[1] + pad);
      q[8] = down(a.box.lo[2] - pad); q[9] = up(a.box.hi[2] + pad);
      q[10] = down(c.box.lo[2] - pad); q[11] = up(c.box.hi[2] + pad);
      const int ca = a.left < 0 ? leaf_code(a) : gpu_index[n.left];
      const int cc = c.left < 0 ? leaf_code(c) : gpu_index[n.right];
      std::memcpy(&q[12], &ca, 4);
      std::memcpy(&q[13], &cc, 4);
    }
  }
  // 4-wide quantized nodes: the binary tree's subtrees are spread over at
  // most four child slots per node so as to minimise the surface-area cost
  // (dynamic programming over "subtree of n in k slots", k = 1..4)
  {
    const size_t NB = B.nodes.size();
    const double kCn = 1.0, kCt = 0.4;   // 4-wide node visit vs triangle test (relative cost)
    std::vector<double> f(NB * 5, 0.0);  // f[n*5+k]: cost of n's subtree in <= k slots
    std::vector<int8_t> sp(NB * 5, 0);   // split of k slots: i to the left child (0: use k-1)
    std::vector<int8_t> gi(NB, 1);       // best left share when n is a 4-wide node
    // children after parents in B.nodes: a reverse sweep sees children first
    for (size_t t = NB; t-- > 0;) {
      const BNode& n = B.nodes[t];
      const double A = n.box.area();
      if (n.left < 0) {
        for (int k = 1; k <= 4; ++k) f[t * 5 + k] = kCt * A * n.count;
        continue;
      }
      const size_t L = (size_t)n.left, R = (size_t)n.right;
      double best = 1e300;
      for (int i = 1; i <= 3; ++i) {
        const double c = f[L * 5 + i] + f[R * 5 + 4 - i];
        if (c < best) {
          best = c;
          gi[t] = (int8_t)i;
        }
      }
      f[t * 5 + 1] = kCn * A + best;  // n as one 4-wide node
      for (int k = 2; k <= 4; ++k) {
        double b2 = f[t * 5 + k - 1];
        int8_t choice = 0;
        for (int i = 1; i <= k - 1; ++i) {
          const double c = f[L * 5 + i] + f[R * 5 + k - i];
          if (c < b2) {
            b2 = c;
            choice = (int8_t)i;
          }
        }
        f[t * 5 + k] = b2;
        sp[t * 5 + k] = choice;
      }
    }
    std::function<void(int, int, std::vector<int>&)> collect = [&](int n, int k, std::vector<int>& out) {
      while (k > 1 && B.nodes[n].left >= 0 && sp[(size_t)n * 5 + k] == 0) --k;
      if (k == 1 || B.nodes[n].left < 0) {
        out.push_back(n);
        return;
      }
      const int i = sp[(size_t)n * 5 + k];
      collect(B.nodes[n].left, i, out);
      collect(B.nodes[n].right, k - i, out);
    };
    std::vector<uint32_t>& out = s.nodes4;
    out.clear();
    struct Item {
      int bnode;
      uint32_t slot;
    };
    std::vector<Item> work;
    auto alloc = [&]() {
      out.resize(out.size() + 16, 0u);
      return (uint32_t)(out.size() / 16 - 1);
    };
    work.push_back({0, alloc()});
    while (!work.empty()) {
      const Item it = work.back();
      work.pop_back();
      std::vector<int> ch;
      const BNode& root = B.nodes[it.bnode];
      if (root.left < 0) {
        ch.push_back(it.bnode);
      } else {
        const int i = gi[(size_t)it.bnode];
        collect(root.left, i, ch);
        collect(root.right, 4 - i, ch);
      }
      Box u;
      u.reset();
      std::vector<Box> cb(ch.size());
      for (size_t i = 0; i < ch.size(); ++i) {
        cb[i] = B.nodes[ch[i]].box;
        for (int k = 0; k < 3; ++k) {
          cb[i].lo[k] -= pad;
          cb[i].hi[k] += pad;
        }
        u.grow(cb[i]);
      }
      ScaleQuantizer qa[3];
      for (int k = 0; k < 3; ++k) qa[k] = make_scale_axis(u.lo[k], u.hi[k]);
      uint32_t w[16] = {0};
      for (int k = 0; k < 3; ++k) {
        std::memcpy(&w[k], &qa[k].p, 4);
        const float s15 = qa[k].s * 32768.0f;  // exact: a power-of-two factor
        std::memcpy(&w[k == 0 ? 3 : 13 + k], &s15, 4);
      }
      for (size_t i = 0; i < ch.size(); ++i) {
        const BNode& c = B.nodes[ch[i]];
        int ref;
        if (c.left < 0) {
          ref = leaf_code(c);
        } else {
          const uint32_t slot = alloc();
          ref = (int)slot;
          work.push_back({ch[i], slot});
        }
        std::memcpy(&w[4 + i], &ref, 4);
        for (int k = 0; k < 3; ++k) {
          w[8 + 2 * k] |= q_lo(qa[k], cb[i].lo[k]) << (8 * i);
          w[9 + 2 * k] |= q_hi(qa[k], cb[i].hi[k]) << (8 * i);
        }
      }
      // Empty slots: an inverted box (lower code 255, upper code 0 on every
      // axis; its near plane lies 255 codes past its far plane whatever the
      // ray's direction), so the node test needs no child count; its link
      // repeats child 0, so even a hit would only revisit a real child.
      for (size_t i = ch.size(); i < 4; ++i) {
        w[4 + i] = w[4];
        for (int k = 0; k < 3; ++k) w[8 + 2 * k] |= 255u << (8 * i);
      }
      std::memcpy(&out[16 * (size_t)it.slot], w, sizeof(w));
    }
    s.n_nodes4 = (uint32_t)(out.size() / 16);
  }
  // 8-wide quantized nodes: the same dynamic programming over at most eight
  // child slots, then the children assigned to slots by octant
  {
    const size_t NB = B.nodes.size();
    const double kCn = 1.0, kCt = 0.4;
    std::vector<double> f(NB * 9, 0.0);
    std::vector<int8_t> sp(NB * 9, 0);
    std::vector<int8_t> gi(NB, 1);
    for (size_t t = NB; t-- > 0;) {
      const BNode& n = B.nodes[t];
      const double A = n.box.area();
      if (n.left < 0) {
        for (int k = 1; k <= 8; ++k) f[t * 9 + k] = kCt * A * n.count;
        continue;
      }
      const size_t L = (size_t)n.left, R = (size_t)n.right;
      double best = 1e300;
      for (int i = 1; i <= 7; ++i) {
        const double c = f[L * 9 + i] + f[R * 9 + 8 - i];
        if (c < best) {
          best = c;
          gi[t] = (int8_t)i;
        }
      }
      f[t * 9 + 1] = kCn * A + best;  // n as one 8-wide node
      for (int k = 2; k <= 8; ++k) {
        double b2 = f[t * 9 + k - 1];
        int8_t choice = 0;
        for (int i = 1; i <= k - 1; ++i) {
          const double c = f[L * 9 + i] + f[R * 9 + k - i];
          if (c < b2) {
            b2 = c;
            choice = (int8_t)i;
          }
        }
        f[t * 9 + k] = b2;
        sp[t * 9 + k] = choice;
      }
    }
    std::function<void(int, int, std::vector<int>&)> collect = [&](int n, int k, std::vector<int>& out) {
      while (k > 1 && B.nodes[n].left >= 0 && sp[(size_t)n * 9 + k] == 0) --k;
      if (k == 1 || B.nodes[n].left < 0) {
        out.push_back(n);
        return;
      }
      const int i = sp[(size_t)n * 9 + k];
      collect(B.nodes[n].left, i, out);
      collect(B.nodes[n].right, k - i, out);
    };
    std::vector<uint32_t>& out = s.nodes8;
    out.clear();
    struct Item {
      int bnode;
      uint32_t slot;
    };
    std::vector<Item> work;
    auto alloc = [&]() {
      out.resize(out.size() + 24, 0u);
      return (uint32_t)(out.size() / 24 - 1);
    };
    work.push_back({0, alloc()});
    while (!work.empty()) {
      const Item it = work.back();
      work.pop_back();
      std::vector<int> ch;
      const BNode& root = B.nodes[it.bnode];
      if (root.left < 0) {
        ch.push_back(it.bnode);
      } else {
        const int i = gi[(size_t)it.bnode];
        collect(root.left, i, ch);
        collect(root.right, 8 - i, ch);
      }
      Box u;
      u.reset();
      std::vector<Box> cb(ch.size());
      for (size_t i = 0; i < ch.size(); ++i) {
        cb[i] = B.nodes[ch[i]].box;
        for (int k = 0; k < 3; ++k) {
          cb[i].lo[k] -= pad;
          cb[i].hi[k] += pad;
        }
        u.grow(cb[i]);
      }
      // Slot j takes the child whose centre lies most towards the octant
      // that is positive on the axes of j's set bits and negative on the
      // others: a ray with direction sign bits sgn (bit set = negative)
      // then meets the children roughly front to back in the order of
      // (slot ^ sgn).  Greedy assignment of the highest remaining
      // (child, slot) score.
      int slot_of[8];
      {
        double score[8][8];
        for (size_t i = 0; i < ch.size(); ++i)
          for (int j = 0; j < 8; ++j) {
            double sc = 0.0;
            for (int k = 0; k < 3; ++k) {
              const double off = 0.5 * (cb[i].lo[k] + cb[i].hi[k]) - 0.5 * (u.lo[k] + u.hi[k]);
              sc += ((j >> k) & 1) ? off : -off;
            }
            score[i][j] = sc;
          }
        bool child_done[8] = {false}, slot_used[8] = {false};
        for (size_t round = 0; round < ch.size(); ++round) {
          double best = -1e300;
          int bi = -1, bj = -1;
          for (size_t i = 0; i < ch.size(); ++i)
            for (int j = 0; j < 8; ++j)
              if (!child_done[i] && !slot_used[j] && score[i][j] > best) {
                best = score[i][j];
                bi = (int)i;
                bj = j;
              }
          child_done[bi] = true;
          slot_used[bj] = true;
          slot_of[bi] = bj;
        }
      }
      Quantizer qa[3];
      for (int k = 0; k < 3; ++k) qa[k] = make_axis(u.lo[k], u.hi[k]);
      uint32_t w[24] = {0};
      for (int k = 0; k < 3; ++k) std::memcpy(&w[k], &qa[k].p, 4);
      uint32_t valid = 0;
      for (size_t i = 0; i < ch.size(); ++i) valid |= 1u << slot_of[i];
      w[3] = (uint32_t)qa[0].e | ((uint32_t)qa[1].e << 8) | ((uint32_t)qa[2].e << 16) | (valid << 24);
      for (size_t i = 0; i < ch.size(); ++i) {
        const BNode& c = B.nodes[ch[i]];
        const int j = slot_of[i];
        int ref;
        if (c.left < 0) {
          ref = leaf_code(c);
        } else {
          const uint32_t slot = alloc();
          ref = (int)slot;
          work.push_back({ch[i], slot});
        }
        std::memcpy(&w[16 + j], &ref, 4);
        for (int k = 0; k < 3; ++k) {
          w[4 + 4 * k + j / 4] |= q_lo(qa[k], cb[i].lo[k]) << (8 * (j % 4));
          w[6 + 4 * k + j / 4] |= q_hi(qa[k], cb[i].hi[k]) << (8 * (j % 4));
        }
      }
      std::memcpy(&out[24 * (size_t)it.slot], w, sizeof(w));
    }
    s.n_nodes8 = (uint32_t)(out.size() / 24);
  }
  // triangles in leaf order
  s.tris.assign(12 * (size_t)n_tri, 0.0f);
  s.orig_to_internal.assign(n_tri, 0);
  if (nrm) s.vnrm.assign(12 * (size_t)n_tri, 0.0f);
  for (uint32_t i = 0; i < n_tri; ++i) {
    const uint32_t t = B.order[i];
    s.orig_to_internal[t] = i;
    float* q = &s.tris[12 * (size_t)i];
    for (int j = 0; j < 3; ++j) {
      const uint32_t v = idx[3 * t + j];
      q[4 * j + 0] = pos[3 * v + 0];
      q[4 * j + 1] = pos[3 * v + 1];
      q[4 * j + 2] = pos[3 * v + 2];
      if (nrm) {
        float* m = &s.vnrm[12 * (size_t)i + 4 * j];
        m[0] = nrm[3 * v];
        m[1] = nrm[3 * v + 1];
        m[2] = nrm[3 * v + 2];
      }
    }
    q[3] = bits_f(t);
    q[7] = bits_f(tri_seg[t]);
  }
  // per-segment triangle lists (increasing original id) and area CDFs
  s.seg_begin.assign(n_seg + 1, 0);
  for (uint32_t t = 0; t < n_tri; ++t) s.seg_begin[tri_seg[t] + 1]++;
  for (uint32_t k = 0; k < n_seg; ++k) s.seg_begin[k + 1] += s.seg_begin[k];
  s.seg_tris.assign(n_tri, 0);
  s.tri_cdf.assign(n_tri, 0.0);
  s.seg_area.assign(n_seg, 0.0);
  std::vector<uint32_t> fill(s.seg_begin.begin(), s.seg_begin.end() - 1);
  std::vector<uint32_t> orig_list(n_tri);
  for (uint32_t t = 0; t < n_tri; ++t) orig_list[fill[tri_seg[t]]++] = t;
  for (uint32_t k = 0; k < n_seg; ++k) {
    double acc = 0.0;
    for (uint32_t j = s.seg_begin[k]; j < s.seg_begin[k + 1]; ++j) {
      acc = acc + area[orig_list[j]];
      s.tri_cdf[j] = acc;
      s.seg_tris[j] = s.orig_to_internal[orig_list[j]];
    }
    s.seg_area[k] = acc;
  }
  if (s.depth + 2 > 64) {
    *err = "BVH deeper than the traversal stack";
    return false;
  }
  return true;
}

}  // namespace ipt
