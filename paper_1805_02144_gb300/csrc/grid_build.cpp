// Icosahedral geodesic Voronoi grid and finite-volume operator tables.
//
// Sec. 2 of the paper discretises the shallow-water equations by finite
// volumes on the control volumes (Voronoi cells) around the N_g = 10*4^l + 2
// nodes of a level-l geodesic grid and writes the operators as sparse
// matrices (Eqs. eq:sweqsinv, eq:vort, eq:swdis).  The grid and operators here:
//   * level 0: icosahedron with vertices at the poles and two rings of five at
//     latitude +-atan(1/2), the southern ring rotated by 36 degrees;
//   * each refinement splits every triangle in four at the normalised edge
//     midpoints (a+b)/|a+b|;
//   * Voronoi vertices are triangle circumcentres (b-a)x(c-a)/|..|;
//   * per directed edge i->j: l_e (Voronoi edge arc length), d_e (node arc
//     distance), m_e (Voronoi edge midpoint), nu_e = (x_j-x_i)/|x_j-x_i|,
//     t_e = m_e x nu_e; A_i = sum of the spherical triangles (x_i, c1, c2)
//     (Oosterom-Strackee formula);
//   * edge values psi_e = (psi(c1) + psi(c2))/2 with psi(c) the barycentric
//     interpolation at the flat-triangle circumcentre (trapezoid rule along the
//     Voronoi edge, exact for linear fields);
//   * (G psi)_i = P_i (1/A_i) sum l nu (psi_e - psi_i), (D.q)_i = (1/A_i) sum
//     l nu.q_e, (V.u)_i = (1/A_i) sum l t.u_e, (L psi)_i = (1/A_i) sum
//     (l/d)(psi_j - psi_i).
// Every edge-value operator has the one-ring stencil {i} U N(i), so each is
// stored as per-slot coefficients plus a diagonal.  Cells are finally sorted
// along a 3-D Hilbert curve (Skilling's transpose construction) so that the
// one-ring of a cell is close in memory.
#include "grid_build.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>
#include <unordered_map>

namespace swe {
namespace {

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return (1.0 / norm(a)) * a; }
inline double arc(V3 a, V3 b) { return std::atan2(norm(cross(a, b)), dot(a, b)); }
inline double tri_solid_angle(V3 a, V3 b, V3 c) {
  double num = std::fabs(dot(a, cross(b, c)));
  double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
  return 2.0 * std::atan2(num, den);
}
inline uint64_t ekey(int a, int b) {
  uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
  return ((uint64_t)hi << 32) | lo;
}
inline uint64_t dkey(int a, int b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; }

struct Tri {
  int v[3];
};

void icosahedron(std::vector<V3>& p, std::vector<Tri>& t) {
  const double s = 1.0 / std::sqrt(5.0), c = 2.0 / std::sqrt(5.0);
  const double pi = 3.14159265358979323846;
  p.clear();
  p.push_back({0.0, 0.0, 1.0});
  for (int k = 0; k < 5; ++k) {
    double lon = 2.0 * pi * k / 5.0;
    p.push_back({c * std::cos(lon), c * std::sin(lon), s});
  }
  for (int k = 0; k < 5; ++k) {
    double lon = 2.0 * pi * k / 5.0 + pi / 5.0;
    p.push_back({c * std::cos(lon), c * std::sin(lon), -s});
  }
  p.push_back({0.0, 0.0, -1.0});
  t.clear();
  for (int k = 0; k < 5; ++k) {
    int k1 = (k + 1) % 5;
    t.push_back({{0, 1 + k, 1 + k1}});
    t.push_back({{1 + k, 6 + k, 1 + k1}});
    t.push_back({{1 + k1, 6 + k, 6 + k1}});
    t.push_back({{11, 6 + k1, 6 + k}});
  }
  for (Tri& f : t) {  // counter-clockwise seen from outside
    V3 a = p[f.v[0]], b = p[f.v[1]], cc = p[f.v[2]];
    if (dot(cross(b - a, cc - a), a + b + cc) < 0) std::swap(f.v[1], f.v[2]);
  }
}

// One refinement.  gen[v] is the generation index of node v (see
// build_host_grid); the new midpoints are numbered here in the order they are
// first met, and their generation indices follow the ascending
// (smaller, larger) generation indices of their parent edges.
void refine(std::vector<V3>& p, std::vector<Tri>& t, std::vector<int32_t>& gen) {
  std::unordered_map<uint64_t, int> mid;
  mid.reserve(t.size() * 2);
  std::vector<std::array<int32_t, 3>> parents;  // (lower gen, upper gen, node)
  auto midpoint = [&](int a, int b) {
    uint64_t k = ekey(a, b);
    auto it = mid.find(k);
    if (it != mid.end()) return it->second;
    int id = (int)p.size();
    p.push_back(unit(p[a] + p[b]));
    mid.emplace(k, id);
    parents.push_back({std::min(gen[a], gen[b]), std::max(gen[a], gen[b]), id});
    return id;
  };
  std::vector<Tri> out;
  out.reserve(t.size() * 4);
  for (const Tri& f : t) {
    int a = f.v[0], b = f.v[1], c = f.v[2];
    int ab = midpoint(a, b), bc = midpoint(b, c), ca = midpoint(c, a);
    out.push_back({{a, ab, ca}});
    out.push_back({{ab, b, bc}});
    out.push_back({{ca, bc, c}});
    out.push_back({{ab, bc, ca}});
  }
  t.swap(out);
  const int32_t nv = (int32_t)gen.size();
  std::sort(parents.begin(), parents.end());
  gen.resize(p.size());
  for (size_t r = 0; r < parents.size(); ++r) gen[parents[r][2]] = nv + (int32_t)r;
}

// Skilling's transpose form of the Hilbert index (J. Skilling, "Programming
// the Hilbert curve", AIP Conf. Proc. 707, 2004), 3 axes of `bits` bits.
uint64_t hilbert3(uint32_t X[3], int bits) {
  const int n = 3;
  uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    uint32_t P = Q - 1;
    for (int i = 0; i < n; ++i) {
      if (X[i] & Q) {
        X[0] ^= P;
      } else {
        uint32_t tt = (X[0] ^ X[i]) & P;
        X[0] ^= tt;
        X[i] ^= tt;
      }
    }
  }
  for (int i = 1; i < n; ++i) X[i] ^= X[i - 1];
  uint32_t tt = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[n - 1] & Q) tt ^= Q - 1;
  for (int i = 0; i < n; ++i) X[i] ^= tt;
  uint64_t key = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int i = 0; i < n; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
  return key;
}

}  // namespace

int build_host_grid(int level, double radius, bool reorder, HostGrid& g, const char** err) {
  if (level < 0 || level > 10) {
    *err = "level must be in [0, 10]";
    return -1;
  }
  std::vector<V3> P;
  std::vector<Tri> T;
  icosahedron(P, T);
  // generation index: the 12 icosahedron nodes in the order above, then per
  // refinement the new midpoints by ascending (smaller, larger) generation
  // index of the edge they split
  std::vector<int32_t> gen(P.size());
  std::iota(gen.begin(), gen.end(), 0);
  for (int l = 0; l < level; ++l) refine(P, T, gen);
  const int ng = (int)P.size();
  const int nt = (int)T.size();

  // directed edge -> triangle on its left; circumcentres
  std::unordered_map<uint64_t, int> left;
  left.reserve((size_t)nt * 3 * 2);
  std::vector<V3> cc(nt);
  std::vector<std::array<double, 3>> lam(nt);
  std::vector<int> deg(ng, 0);
  for (int t = 0; t < nt; ++t) {
    const int* v = T[t].v;
    for (int e = 0; e < 3; ++e) {
      left.emplace(dkey(v[e], v[(e + 1) % 3]), t);
      deg[v[e]]++;
    }
    V3 a = P[v[0]], b = P[v[1]], c = P[v[2]];
    cc[t] = unit(cross(b - a, c - a));
    double la = dot(b - c, b - c), lb = dot(c - a, c - a), lc = dot(a - b, a - b);
    double wa = la * (lb + lc - la), wb = lb * (lc + la - lb), wc = lc * (la + lb - lc);
    double sw = wa + wb + wc;
    lam[t] = {wa / sw, wb / sw, wc / sw};
  }
  for (int i = 0; i < ng; ++i)
    if (deg[i] != 5 && deg[i] != 6) {
      *err = "unexpected vertex degree";
      return -1;
    }

  // counter-clockwise neighbour ring of every node
  std::vector<int32_t> ring((size_t)kSlots * ng, -1);
  {
    std::vector<int> first(ng, -1);
    for (int t = 0; t < nt; ++t)
      for (int e = 0; e < 3; ++e) {
        int a = T[t].v[e], b = T[t].v[(e + 1) % 3];
        if (first[a] < 0) first[a] = b;
      }
    for (int i = 0; i < ng; ++i) {
      int j = first[i];
      for (int k = 0; k < deg[i]; ++k) {
        ring[(size_t)i * kSlots + k] = j;
        const Tri& f = T[left.at(dkey(i, j))];
        int nx = -1;  // third vertex of the triangle left of i->j is the next CCW neighbour
        for (int e = 0; e < 3; ++e)
          if (f.v[e] != i && f.v[e] != j) nx = f.v[e];
        j = nx;
      }
      if (j != first[i]) {
        *err = "neighbour ring does not close";
        return -1;
      }
    }
  }

  // areas first (coefficients carry 1/A_i)
  std::vector<double> area(ng, 0.0);
  for (int i = 0; i < ng; ++i) {
    double s = 0.0;
    for (int k = 0; k < deg[i]; ++k) {
      int j = ring[(size_t)i * kSlots + k];
      V3 c1 = cc[left.at(dkey(i, j))], c2 = cc[left.at(dkey(j, i))];
      s += tri_solid_angle(P[i], c1, c2);
    }
    area[i] = radius * radius * s;
  }

  // per-cell slot coefficients in generation order
  std::vector<double> wl((size_t)kSlots * ng, 0.0), wld(ng, 0.0);
  std::vector<double> nc((size_t)3 * kSlots * ng, 0.0), ndd((size_t)3 * ng, 0.0),
      sdg((size_t)3 * ng, 0.0);
  std::vector<double> vc((size_t)3 * kSlots * ng, 0.0), vd((size_t)3 * ng, 0.0);
  for (int i = 0; i < ng; ++i) {
    const int32_t* rg = &ring[(size_t)i * kSlots];
    auto slot_of = [&](int v) {
      if (v == i) return -1;
      for (int k = 0; k < deg[i]; ++k)
        if (rg[k] == v) return k;
      return -2;
    };
    const double inva = 1.0 / area[i];
    for (int k = 0; k < deg[i]; ++k) {
      int j = rg[k];
      int tl = left.at(dkey(i, j)), tr = left.at(dkey(j, i));
      V3 c1 = cc[tl], c2 = cc[tr];
      double le = radius * arc(c1, c2);
      double de = radius * arc(P[i], P[j]);
      V3 me = unit(c1 + c2);
      V3 nu = unit(P[j] - P[i]);
      V3 te = cross(me, nu);
      double gnu[3] = {le * nu.x * inva, le * nu.y * inva, le * nu.z * inva};
      double gte[3] = {le * te.x * inva, le * te.y * inva, le * te.z * inva};
      for (int c = 0; c < 3; ++c) sdg[(size_t)c * ng + i] += gnu[c];
      double w = le / de * inva;
      wl[(size_t)k * ng + i] += w;
      wld[i] -= w;
      for (int side = 0; side < 2; ++side) {
        int t = side == 0 ? tl : tr;
        for (int e = 0; e < 3; ++e) {
          int v = T[t].v[e];
          double wt = 0.5 * lam[t][e];
          int s = slot_of(v);
          if (s == -2) {
            *err = "edge-value stencil leaves the one-ring";
            return -1;
          }
          for (int c = 0; c < 3; ++c) {
            if (s < 0) {
              ndd[(size_t)c * ng + i] += gnu[c] * wt;
              vd[(size_t)c * ng + i] += gte[c] * wt;
            } else {
              nc[((size_t)c * kSlots + s) * ng + i] += gnu[c] * wt;
              vc[((size_t)c * kSlots + s) * ng + i] += gte[c] * wt;
            }
          }
        }
      }
    }
  }

  // structural nonzeros of J: 4 (3 |R1(i)| + |R2(i)|) per cell
  int64_t nA = 0;
  for (int i = 0; i < ng; ++i) {
    int r2[64];
    int n2 = 0;
    auto add = [&](int v) {
      for (int q = 0; q < n2; ++q)
        if (r2[q] == v) return;
      r2[n2++] = v;
    };
    add(i);
    for (int k = 0; k < deg[i]; ++k) add(ring[(size_t)i * kSlots + k]);
    int n1 = n2;
    for (int k = 0; k < deg[i]; ++k) {
      int j = ring[(size_t)i * kSlots + k];
      for (int q = 0; q < deg[j]; ++q) add(ring[(size_t)j * kSlots + q]);
    }
    nA += 4 * (3 * n1 + n2);
  }

  // cell order: Hilbert curve over the unit-cube coordinates, or generation order
  std::vector<int> perm(ng);  // new -> old
  std::iota(perm.begin(), perm.end(), 0);
  if (reorder) {
    const int bits = 21;
    std::vector<uint64_t> key(ng);
    const double sc = (double)((1u << bits) - 1);
    for (int i = 0; i < ng; ++i) {
      uint32_t X[3] = {(uint32_t)std::lround((P[i].x + 1.0) * 0.5 * sc),
                       (uint32_t)std::lround((P[i].y + 1.0) * 0.5 * sc),
                       (uint32_t)std::lround((P[i].z + 1.0) * 0.5 * sc)};
      key[i] = hilbert3(X, bits);
    }
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return key[a] < key[b]; });
  }
  std::vector<int> inv(ng);
  for (int i = 0; i < ng; ++i) inv[perm[i]] = i;

  g.level = level;
  g.ng = ng;
  g.radius = radius;
  g.nA = nA;
  g.xyz.assign((size_t)3 * ng, 0.0);
  g.area.assign(ng, 0.0);
  g.nbr.assign((size_t)kSlots * ng, 0);
  g.wl.assign((size_t)kSlots * ng, 0.0);
  g.wld.assign(ng, 0.0);
  g.nc.assign((size_t)3 * kSlots * ng, 0.0);
  g.vc.assign((size_t)3 * kSlots * ng, 0.0);
  g.ndd.assign((size_t)3 * ng, 0.0);
  g.sdg.assign((size_t)3 * ng, 0.0);
  g.vd.assign((size_t)3 * ng, 0.0);
  g.gen.assign(ng, 0);
  for (int ni = 0; ni < ng; ++ni) {
    int i = perm[ni];
    g.gen[ni] = gen[i];
    g.xyz[ni] = P[i].x;
    g.xyz[(size_t)ng + ni] = P[i].y;
    g.xyz[(size_t)2 * ng + ni] = P[i].z;
    g.area[ni] = area[i];
    g.wld[ni] = wld[i];
    for (int k = 0; k < kSlots; ++k) {
      bool real = k < deg[i];
      g.nbr[(size_t)k * ng + ni] = real ? inv[ring[(size_t)i * kSlots + k]] : ni;
      g.wl[(size_t)k * ng + ni] = wl[(size_t)k * ng + i];
      for (int c = 0; c < 3; ++c) {
        g.nc[((size_t)c * kSlots + k) * ng + ni] = nc[((size_t)c * kSlots + k) * ng + i];
        g.vc[((size_t)c * kSlots + k) * ng + ni] = vc[((size_t)c * kSlots + k) * ng + i];
      }
    }
    for (int c = 0; c < 3; ++c) {
      g.ndd[(size_t)c * ng + ni] = ndd[(size_t)c * ng + i];
      g.sdg[(size_t)c * ng + ni] = sdg[(size_t)c * ng + i];
      g.vd[(size_t)c * ng + ni] = vd[(size_t)c * ng + i];
    }
  }
  // transposed slot tables
  g.wlT.assign((size_t)kSlots * ng, 0.0);
  g.ncT.assign((size_t)3 * kSlots * ng, 0.0);
  g.vcT.assign((size_t)3 * kSlots * ng, 0.0);
  for (int j = 0; j < ng; ++j) {
    for (int k = 0; k < kSlots; ++k) {
      const int i = g.nbr[(size_t)k * ng + j];
      if (i == j) continue;  // pad slot of a pentagon
      int s = -1;
      for (int q = 0; q < kSlots; ++q)
        if (g.nbr[(size_t)q * ng + i] == j) s = q;
      if (s < 0) {
        *err = "neighbour relation is not symmetric";
        return -1;
      }
      g.wlT[(size_t)k * ng + j] = g.wl[(size_t)s * ng + i];
      for (int c = 0; c < 3; ++c) {
        g.ncT[((size_t)c * kSlots + k) * ng + j] = g.nc[((size_t)c * kSlots + s) * ng + i];
        g.vcT[((size_t)c * kSlots + k) * ng + j] = g.vc[((size_t)c * kSlots + s) * ng + i];
      }
    }
  }
  return 0;
}

}  // namespace swe
