// Structural check of the scene builder's wide BVHs, compiled and run on the
// host by tests/test_bvh_cpu.py.  It decodes the nodes on its own and checks
// that, in the 4-wide tree (64-byte nodes: origin, per-axis float scales,
// 8-bit child codes, links) and in the 8-wide tree (96-byte nodes: origin,
// per-axis power-of-two scales, occupied-slot mask, codes, links),
//  * every triangle lies in exactly one leaf,
//  * every child box, p + q * scale per axis evaluated in double, contains
//    the exact bounds of all triangles below that child,
//  * 4-wide empty slots hold inverted boxes and repeat child 0's link.
// Input (binary files): float32 positions (n_vert x 3), uint32 indices
// (n_tri x 3).  Prints "tris_once4 violations4 tris_once8 violations8
// nodes4 depth".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <string>
#include <vector>

#include "ipt_internal.h"

namespace {

struct Bounds {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  void grow(const Bounds& b) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::fmin(lo[k], b.lo[k]);
      hi[k] = std::fmax(hi[k], b.hi[k]);
    }
  }
};

const ipt::HostScene* S;
std::vector<int> seen;
long violations = 0;

float word_f(uint32_t w) {
  float f;
  std::memcpy(&f, &w, 4);
  return f;
}

// bounds of the triangles below link `ref`, checking the subtree on the way
Bounds visit(int ref) {
  Bounds b;
  if (ref < 0) {
    const int v = -ref - 1, first = v >> 3, count = (v & 7) + 1;
    for (int i = first; i < first + count; ++i) {
      if (i < 0 || i >= (int)S->n_tri) {
        ++violations;
        continue;
      }
      ++seen[i];
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          const double x = S->tris[12 * (size_t)i + 4 * j + k];
          b.lo[k] = std::fmin(b.lo[k], x);
          b.hi[k] = std::fmax(b.hi[k], x);
        }
    }
    return b;
  }
  const uint32_t* w = &S->nodes4[16 * (size_t)ref];
  const double p[3] = {word_f(w[0]), word_f(w[1]), word_f(w[2])};
  const double s[3] = {word_f(w[3]) / 32768.0, word_f(w[14]) / 32768.0, word_f(w[15]) / 32768.0};
  for (int i = 0; i < 4; ++i) {
    int link;
    std::memcpy(&link, &w[4 + i], 4);
    uint32_t qlo[3], qhi[3];
    for (int k = 0; k < 3; ++k) {
      qlo[k] = (w[8 + 2 * k] >> (8 * i)) & 0xffu;
      qhi[k] = (w[9 + 2 * k] >> (8 * i)) & 0xffu;
    }
    const bool empty = qlo[0] == 255 && qhi[0] == 0 && qlo[1] == 255 && qhi[1] == 0 && qlo[2] == 255 && qhi[2] == 0;
    if (empty) {
      int first;
      std::memcpy(&first, &w[4], 4);
      if (i == 0 || link != first) ++violations;
      continue;
    }
    const Bounds c = visit(link);
    for (int k = 0; k < 3; ++k)
      if (p[k] + qlo[k] * s[k] > c.lo[k] || p[k] + qhi[k] * s[k] < c.hi[k]) ++violations;
    b.grow(c);
  }
  return b;
}

// the same for the 8-wide tree
Bounds visit8(int ref) {
  Bounds b;
  if (ref < 0) return visit(ref);
  const uint32_t* w = &S->nodes8[24 * (size_t)ref];
  const double p[3] = {word_f(w[0]), word_f(w[1]), word_f(w[2])};
  double s[3];
  for (int k = 0; k < 3; ++k) s[k] = std::ldexp(1.0, (int)((w[3] >> (8 * k)) & 0xffu) - 127);
  const uint32_t valid = w[3] >> 24;
  for (int j = 0; j < 8; ++j) {
    if (!(valid >> j & 1u)) continue;
    int link;
    std::memcpy(&link, &w[16 + j], 4);
    const Bounds c = visit8(link);
    for (int k = 0; k < 3; ++k) {
      const uint32_t qlo = (w[4 + 4 * k + j / 4] >> (8 * (j % 4))) & 0xffu;
      const uint32_t qhi = (w[6 + 4 * k + j / 4] >> (8 * (j % 4))) & 0xffu;
      if (p[k] + qlo * s[k] > c.lo[k] || p[k] + qhi * s[k] < c.hi[k]) ++violations;
    }
    b.grow(c);
  }
  return b;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 5) return 2;
  const uint32_t nv = (uint32_t)std::strtoul(argv[3], nullptr, 10), nt = (uint32_t)std::strtoul(argv[4], nullptr, 10);
  std::vector<float> pos(3 * (size_t)nv);
  std::vector<uint32_t> idx(3 * (size_t)nt), seg(nt, 0);
  std::ifstream(argv[1], std::ios::binary).read(reinterpret_cast<char*>(pos.data()), pos.size() * 4);
  std::ifstream(argv[2], std::ios::binary).read(reinterpret_cast<char*>(idx.data()), idx.size() * 4);
  ipt::HostScene hs;
  std::string err;
  if (!ipt::build_scene(pos.data(), nv, nullptr, idx.data(), nt, seg.data(), 1, &hs, &err)) {
    std::printf("build failed: %s\n", err.c_str());
    return 1;
  }
  S = &hs;
  long once[2] = {0, 0}, viol[2] = {0, 0};
  for (int wide = 0; wide < 2; ++wide) {
    seen.assign(nt, 0);
    violations = 0;
    if (wide == 0) visit(0);
    else if (hs.n_nodes8 > 0) visit8(0);
    for (int v : seen) once[wide] += v == 1;
    viol[wide] = violations;
  }
  std::printf("%ld %ld %ld %ld %u %u\n", once[0], viol[0], once[1], viol[1], hs.n_nodes4, hs.depth);
  return 0;
}
