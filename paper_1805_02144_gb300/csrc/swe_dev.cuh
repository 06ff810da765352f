// Device-side building blocks: operator tables, the two-pass cell stencils of
// F(u), J(u)x and the quadratic part Q(d), and bounded grid-wide barriers.
// The stencils are templated on the real type R of tables, vectors and
// arithmetic: double for the FP64 path, float for the mixed-precision path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace swe {

constexpr int SLOTS = 6;

// Operator tables of one grid in precision R (read-only for the grid's life).
template <typename R>
struct TablesT {
  int ng;
  R nu;           // dissipation coefficient of Eq. eq:niu
  R g;            // gravity
  R two_omega;
  const int32_t* __restrict__ nbr;  // [6][ng]
  const R* __restrict__ nrm;   // [3][ng] unit normals
  const R* __restrict__ wl;    // [6][ng]
  const R* __restrict__ wld;   // [ng]
  const R* __restrict__ nwl;   // [6][ng] -nu wl: the dissipation's Laplacian weights
  const R* __restrict__ nwld;  // [ng]    -nu wld
  const R* __restrict__ nc;    // [3][6][ng]
  const R* __restrict__ ndd;   // [3][ng]
  const R* __restrict__ gdg;   // [3][ng] G diagonal (ndd - sdg of the host tables)
  const R* __restrict__ vc;    // [3][6][ng]
  const R* __restrict__ vd;    // [3][ng]
  const R* __restrict__ area;  // [ng] cell areas A_i (FP64 grids only)
  const R* __restrict__ hs;    // [ng] surface height h_s, or nullptr (none)
  // transposed slot tables (FP64 grids only; see grid_build.h)
  const R* __restrict__ wlT;   // [6][ng]
  const R* __restrict__ ncT;   // [3][6][ng]
  const R* __restrict__ vcT;   // [3][6][ng]
};
using Tables = TablesT<double>;
using TablesF = TablesT<float>;

// Pass-1 outputs per cell: 4 Laplacian planes and 4 scalar/vector planes.
enum StencilMode { MODE_F = 0, MODE_J = 1, MODE_Q = 2 };

// ---------------------------------------------------------------------------
// Loads.  Vectors may be written inside the same persistent launch (basis,
// stage vectors, and in an ensemble launch the states themselves), so they are
// read with plain coherent loads (`ld`).  Operator tables are fixed for the
// grid's life: they are read once per cell and pass through the non-coherent
// path, bypass L1 allocation and are marked first to leave L2, so that L1 and
// L2 keep the gathered vectors.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R ld(const R* p) { return *p; }

__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double ldtab(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
      : "=d"(v) : "l"(p), "l"(l2_evict_first_policy()));
  return v;
}
__device__ __forceinline__ float ldtab(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
      : "=f"(v) : "l"(p), "l"(l2_evict_first_policy()));
  return v;
}
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// Neighbour indices start every stencil's dependent chain (index -> gather)
// and are read by both passes of every J x: they are kept in L2 (evict-last)
// so that the chain starts with an L2 hit; the coefficient tables stream.
__device__ __forceinline__ int ldtabi(const int32_t* p) {
  int v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
      : "=r"(v) : "l"(p), "l"(l2_evict_last_policy()));
  return v;
}

// L psi at cell i for one plane: wld_i psi_i + sum_k wl_k psi_{nbr_k}
template <typename R>
__device__ __forceinline__ R lap_cell(const TablesT<R>& T, int i, const int (&nb)[SLOTS], const R* psi) {
  R acc = ldtab(T.wld + i) * ld(psi + i);
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) acc = fma(ldtab(T.wl + (size_t)k * T.ng + i), ld(psi + nb[k]), acc);
  return acc;
}

// Neighbour indices of a block's own cells [c0, c0 + stride) copied into
// shared memory by a persistent launch: slot k of cell i at
// s[k * stride + (i - c0)].  An empty view (s == nullptr) reads the table in
// global memory.  Staged indices take the L2 round trip off the start of
// every stencil's index -> gather chain.
struct NbrStage {
  const int32_t* s = nullptr;
  int c0 = 0, stride = 0;
};

template <typename R>
__device__ __forceinline__ void load_nbr(const TablesT<R>& T, int i, int (&nb)[SLOTS],
                                         const NbrStage& st = NbrStage()) {
  if (st.s) {
    const int32_t* q = st.s + (i - st.c0);
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) nb[k] = q[k * st.stride];
  } else {
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) nb[k] = ldtabi(T.nbr + (size_t)k * T.ng + i);
  }
}

// The pass-1 planes (4 Laplacian, 4 scalar/vector) are planar, [4][ng], or
// with IL interleaved, [ng][4]: one 16-byte vector per cell, so that a
// neighbour's four values come in one gather.  IL is used by the FP32
// instantiations only; the arithmetic is the same in both layouts.
template <bool IL, typename R>
__device__ __forceinline__ void st_planes(R* base, int ng, int i, const R (&v)[4]) {
  if constexpr (IL) {
    static_assert(sizeof(R) == 4, "interleaved planes are FP32");
    *reinterpret_cast<float4*>(base + 4 * (size_t)i) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) base[(size_t)c * ng + i] = v[c];
  }
}
template <bool IL, typename R>
__device__ __forceinline__ void ld_planes(const R* base, int ng, int i, R (&v)[4]) {
  if constexpr (IL) {
    static_assert(sizeof(R) == 4, "interleaved planes are FP32");
    const float4 q = *reinterpret_cast<const float4*>(base + 4 * (size_t)i);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = ld(base + (size_t)c * ng + i);
  }
}

// Pass 1 of a stencil at cell i.  Writes four Laplacian planes to Lout and
// the scalar and vector planes to sq (4 planes: scalar, vector x, y, z):
//   MODE_F: x = u.          L u (4), E = |u|^2/2 + g (h + h_s), q = u h
//   MODE_J: x = sx * xraw.  L x (4), s = u.x_u + g x_h,  q = x_u h + u x_h
//   MODE_Q: x = d.          -,       E = |d_u|^2/2,      q = d_u d_h
template <int MODE, typename R, bool IL = false>
__device__ __forceinline__ void pass1_cell(const TablesT<R>& T, int i, const R* x, R sx, const R* u,
                                           R* Lout, R* sq, const NbrStage& st = NbrStage()) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, i, nb, st);
  R xv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) xv[c] = ld(x + (size_t)c * ng + i);
  if (MODE != MODE_Q) {
    R lv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      R lx = lap_cell(T, i, nb, x + (size_t)c * ng);
      lv[c] = (MODE == MODE_J) ? sx * lx : lx;
    }
    st_planes<IL>(Lout, ng, i, lv);
  }
  R sv[4];
  if (MODE == MODE_J) {
#pragma unroll
    for (int c = 0; c < 4; ++c) xv[c] *= sx;
    R uv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) uv[c] = ld(u + (size_t)c * ng + i);
    sv[0] = fma(uv[0], xv[0], fma(uv[1], xv[1], fma(uv[2], xv[2], T.g * xv[3])));
#pragma unroll
    for (int c = 0; c < 3; ++c) sv[1 + c] = fma(xv[c], uv[3], uv[c] * xv[3]);
  } else if (MODE == MODE_F) {
    const R hsurf = T.hs ? ld(T.hs + i) : R(0);  // E = |u|^2/2 + g (h + h_s)
    sv[0] = fma(R(0.5), fma(xv[0], xv[0], fma(xv[1], xv[1], xv[2] * xv[2])), T.g * (xv[3] + hsurf));
#pragma unroll
    for (int c = 0; c < 3; ++c) sv[1 + c] = xv[c] * xv[3];
  } else {
    sv[0] = R(0.5) * fma(xv[0], xv[0], fma(xv[1], xv[1], xv[2] * xv[2]));
#pragma unroll
    for (int c = 0; c < 3; ++c) sv[1 + c] = xv[c] * xv[3];
  }
  st_planes<IL>(sq, ng, i, sv);
}

// Fused IOM2 orthogonalisation and pass 1 (MODE_J) at cell i.  z is A r_j
// of the raw basis vector r_j (complete on every cell) and zs the factor that
// makes zs z the column's dt A v_j; r_j and r_m are the raw basis vectors j
// and j-1 with their Laplacian planes Lj, Lm; aj, am the window coefficients
// with the basis scales folded in (am = 0 and r_m, Lm unused for j = 0):
//   z' = zs z - aj r_j - am r_m                       -> rnew (own cell)
//   L z' = zs L z - aj L r_j - am L r_m               -> Lnew (L is linear)
//   s', q' of z'                                      -> sq
// and returns |z'|^2 of the cell.  No value of z' is gathered, so rnew may be
// written while neighbours still read z.
template <typename R, bool IL = false>
__device__ __forceinline__ R orth_pass1_cell(const TablesT<R>& T, int i, const R* z, R zs, const R* rj,
                                             const R* rm, R aj, R am, const R* Lj, const R* Lm,
                                             R* rnew, R* Lnew, const R* u, R* sq,
                                             const NbrStage& st = NbrStage()) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, i, nb, st);
  R Ljv[4], Lmv[4] = {R(0), R(0), R(0), R(0)}, lzv[4];
  ld_planes<IL>(Lj, ng, i, Ljv);
  if (rm) ld_planes<IL>(Lm, ng, i, Lmv);
  R zp[4], nrm = R(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const size_t e = (size_t)c * ng + i;
    R v = fma(-aj, ld(rj + e), zs * ld(z + e));
    R lz = fma(-aj, Ljv[c], zs * lap_cell(T, i, nb, z + (size_t)c * ng));
    if (rm) {
      v = fma(-am, ld(rm + e), v);
      lz = fma(-am, Lmv[c], lz);
    }
    zp[c] = v;
    rnew[e] = v;
    lzv[c] = lz;
    nrm = fma(v, v, nrm);
  }
  st_planes<IL>(Lnew, ng, i, lzv);
  R uv[4], sv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) uv[c] = ld(u + (size_t)c * ng + i);
  sv[0] = fma(uv[0], zp[0], fma(uv[1], zp[1], fma(uv[2], zp[2], T.g * zp[3])));
#pragma unroll
  for (int c = 0; c < 3; ++c) sv[1 + c] = fma(zp[c], uv[3], uv[c] * zp[3]);
  st_planes<IL>(sq, ng, i, sv);
  return nrm;
}

// Pass 2 of a stencil at cell i: out[4] = F(u), J(u)x or Q(d) at cell i.
//   x: the same vector as pass 1 (F: u, J: raw x with scale sx, Q: d)
//   Lp, sq: the planes pass 1 wrote (Laplacian, scalar + vector)
//   aux (MODE_J only): [eta, P_x, P_y, P_z] of the linearisation state,
//   eta = V u + f, P = n x u.
template <int MODE, typename R, bool IL = false>
__device__ __forceinline__ void pass2_cell(const TablesT<R>& T, int i, const R* x, R sx, const R* Lp,
                                           const R* sq, const R* aux, R out[4],
                                           const NbrStage& st = NbrStage()) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, i, nb, st);
  // relative vorticity of x: V . x_u
  R vor = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) vor = fma(ldtab(T.vd + (size_t)c * ng + i), ld(x + (size_t)c * ng + i), vor);
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    const int j = nb[k];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      vor = fma(ldtab(T.vc + ((size_t)c * SLOTS + k) * ng + i), ld(x + (size_t)c * ng + j), vor);
  }
  // gradient of the scalar plane (before projection) and divergence of the vector planes
  R sqi[4];
  ld_planes<IL>(sq, ng, i, sqi);
  R gr[3], dv = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gr[c] = ldtab(T.gdg + (size_t)c * ng + i) * sqi[0];
    dv = fma(ldtab(T.ndd + (size_t)c * ng + i), sqi[1 + c], dv);
  }
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    R sqj[4];
    ld_planes<IL>(sq, ng, nb[k], sqj);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R w = ldtab(T.nc + ((size_t)c * SLOTS + k) * ng + i);
      gr[c] = fma(w, sqj[0], gr[c]);
      dv = fma(w, sqj[1 + c], dv);
    }
  }
  R n0 = ldtab(T.nrm + i), n1 = ldtab(T.nrm + ng + i), n2 = ldtab(T.nrm + 2 * (size_t)ng + i);
  R ngr = fma(n0, gr[0], fma(n1, gr[1], n2 * gr[2]));
  gr[0] = fma(-n0, ngr, gr[0]);
  gr[1] = fma(-n1, ngr, gr[1]);
  gr[2] = fma(-n2, ngr, gr[2]);
  R xo[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) xo[c] = ld(x + (size_t)c * ng + i);
  R nx0 = n1 * xo[2] - n2 * xo[1];
  R nx1 = n2 * xo[0] - n0 * xo[2];
  R nx2 = n0 * xo[1] - n1 * xo[0];
  if (MODE == MODE_J) {
    vor *= sx;
    nx0 *= sx;
    nx1 *= sx;
    nx2 *= sx;
    R eta = ld(aux + i);
    R p0 = ld(aux + (size_t)ng + i), p1 = ld(aux + 2 * (size_t)ng + i), p2 = ld(aux + 3 * (size_t)ng + i);
    out[0] = -fma(vor, p0, fma(eta, nx0, gr[0]));
    out[1] = -fma(vor, p1, fma(eta, nx1, gr[1]));
    out[2] = -fma(vor, p2, fma(eta, nx2, gr[2]));
    out[3] = -dv;
  } else if (MODE == MODE_F) {
    R eta = fma(T.two_omega, n2, vor);
    out[0] = -fma(eta, nx0, gr[0]);
    out[1] = -fma(eta, nx1, gr[1]);
    out[2] = -fma(eta, nx2, gr[2]);
    out[3] = -dv;
  } else {
    out[0] = -fma(vor, nx0, gr[0]);
    out[1] = -fma(vor, nx1, gr[1]);
    out[2] = -fma(vor, nx2, gr[2]);
    out[3] = -dv;
  }
  if (MODE != MODE_Q) {  // dissipation -nu L (L x) on every variable: (nwl, nwld) hold -nu L
    R Lv[4];
    ld_planes<IL>(Lp, ng, i, Lv);
    const R wd = ldtab(T.nwld + i);
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = fma(wd, Lv[c], out[c]);
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) {
      ld_planes<IL>(Lp, ng, nb[k], Lv);
      const R w = ldtab(T.nwl + (size_t)k * ng + i);
#pragma unroll
      for (int c = 0; c < 4; ++c) out[c] = fma(w, Lv[c], out[c]);
    }
  }
}

// aux = [eta, n x u] of a linearisation state u at cell i.
template <typename R>
__device__ __forceinline__ void aux_cell(const TablesT<R>& T, int i, const R* u, R* aux) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, i, nb);
  R vor = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) vor = fma(ldtab(T.vd + (size_t)c * ng + i), ld(u + (size_t)c * ng + i), vor);
#pragma unroll
  for (int k = 0; k < SLOTS; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      vor = fma(ldtab(T.vc + ((size_t)c * SLOTS + k) * ng + i), ld(u + (size_t)c * ng + nb[k]), vor);
  R n0 = ldtab(T.nrm + i), n1 = ldtab(T.nrm + ng + i), n2 = ldtab(T.nrm + 2 * (size_t)ng + i);
  R u0 = ld(u + i), u1 = ld(u + ng + i), u2 = ld(u + 2 * (size_t)ng + i);
  aux[i] = fma(T.two_omega, n2, vor);
  aux[(size_t)ng + i] = n1 * u2 - n2 * u1;
  aux[2 * (size_t)ng + i] = n2 * u0 - n0 * u2;
  aux[3 * (size_t)ng + i] = n0 * u1 - n1 * u0;
}

// ---------------------------------------------------------------------------
// Transposed stencils (adjoint).  With J x = -(V x_u) P - eta (n x x_u)
// - G s(x) - nu L L x, continuity -D q(x) - nu L L x_h, where
// s(x) = u.x_u + g x_h, q(x) = x_u h + u x_h, P = n x u, eta = V u + f and
// G = P_n R (P_n = I - n n^T the tangent projection), the transpose is
//   xbar_u,d = -(V_d^T a) + eta (n x lam_u) + u sbar + h qbar
//   xbar_h   = g sbar + u.qbar
//   xbar    += -nu L^T L^T lam                          (each variable)
// with a = P.lam_u, sbar = -sum_c R_c^T (P_n lam_u)_c, qbar_c = -D_c^T lam_h.
// MODE_JT: J(u)^T lam (aux = eta, P of u).
// MODE_QT: (J(x) - J(0))^T lam, the transposed derivative of the quadratic
// part at x: eta = V x without f, no g term, no dissipation (aux of x with
// two_omega = 0).
// ---------------------------------------------------------------------------
enum TransMode { MODE_JT = 0, MODE_QT = 1 };

// Pass 1 at cell i: t planes [a, (P_n lam_u) x 3, L^T lam x 4 (MODE_JT)].
template <int MODE>
__device__ __forceinline__ void pass1T_cell(const Tables& T, int i, const double* lam, const double* aux,
                                            double* t) {
  const int ng = T.ng;
  double lu[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) lu[c] = ld(lam + (size_t)c * ng + i);
  double p0 = ld(aux + (size_t)ng + i), p1 = ld(aux + 2 * (size_t)ng + i), p2 = ld(aux + 3 * (size_t)ng + i);
  t[i] = fma(p0, lu[0], fma(p1, lu[1], p2 * lu[2]));
  double n0 = ldtab(T.nrm + i), n1 = ldtab(T.nrm + ng + i), n2 = ldtab(T.nrm + 2 * (size_t)ng + i);
  double nl = fma(n0, lu[0], fma(n1, lu[1], n2 * lu[2]));
  t[(size_t)ng + i] = fma(-n0, nl, lu[0]);
  t[2 * (size_t)ng + i] = fma(-n1, nl, lu[1]);
  t[3 * (size_t)ng + i] = fma(-n2, nl, lu[2]);
  if (MODE == MODE_JT) {
    int nb[SLOTS];
    load_nbr(T, i, nb);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double* psi = lam + (size_t)c * ng;
      double acc = ldtab(T.wld + i) * ld(psi + i);
#pragma unroll
      for (int k = 0; k < SLOTS; ++k) acc = fma(ldtab(T.wlT + (size_t)k * ng + i), ld(psi + nb[k]), acc);
      t[(size_t)(4 + c) * ng + i] = acc;
    }
  }
}

// Pass 2 at cell j: out[4] = (J^T lam)_j (MODE_JT) or ((J(x)-J(0))^T lam)_j
// (MODE_QT).  u: linearisation state (x for MODE_QT); aux: its eta, P.
template <int MODE>
__device__ __forceinline__ void pass2T_cell(const Tables& T, int j, const double* lam, const double* u,
                                            const double* aux, const double* t, double out[4]) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, j, nb);
  double va[3], sb = 0.0, qb[3];
  const double aj = ld(t + j), lhj = ld(lam + 3 * (size_t)ng + j);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    va[c] = ldtab(T.vd + (size_t)c * ng + j) * aj;
    sb = fma(ldtab(T.gdg + (size_t)c * ng + j), ld(t + (size_t)(1 + c) * ng + j), sb);
    qb[c] = ldtab(T.ndd + (size_t)c * ng + j) * lhj;
  }
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    const int i = nb[k];
    const double ai = ld(t + i), lhi = ld(lam + 3 * (size_t)ng + i);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double w = ldtab(T.ncT + ((size_t)c * SLOTS + k) * ng + j);
      va[c] = fma(ldtab(T.vcT + ((size_t)c * SLOTS + k) * ng + j), ai, va[c]);
      sb = fma(w, ld(t + (size_t)(1 + c) * ng + i), sb);
      qb[c] = fma(w, lhi, qb[c]);
    }
  }
  sb = -sb;
  double n0 = ldtab(T.nrm + j), n1 = ldtab(T.nrm + ng + j), n2 = ldtab(T.nrm + 2 * (size_t)ng + j);
  double l0 = ld(lam + j), l1 = ld(lam + (size_t)ng + j), l2 = ld(lam + 2 * (size_t)ng + j);
  double eta = ld(aux + j);
  double uv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) uv[c] = ld(u + (size_t)c * ng + j);
  // eta (n x lam_u)
  double r0 = eta * (n1 * l2 - n2 * l1), r1 = eta * (n2 * l0 - n0 * l2), r2 = eta * (n0 * l1 - n1 * l0);
  out[0] = fma(uv[0], sb, fma(-uv[3], qb[0], r0 - va[0]));
  out[1] = fma(uv[1], sb, fma(-uv[3], qb[1], r1 - va[1]));
  out[2] = fma(uv[2], sb, fma(-uv[3], qb[2], r2 - va[2]));
  out[3] = -fma(uv[0], qb[0], fma(uv[1], qb[1], uv[2] * qb[2]));
  if (MODE == MODE_JT) {
    out[3] = fma(T.g, sb, out[3]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double* psi = t + (size_t)(4 + c) * ng;
      double acc = ldtab(T.wld + j) * ld(psi + j);
#pragma unroll
      for (int k = 0; k < SLOTS; ++k) acc = fma(ldtab(T.wlT + (size_t)k * ng + j), ld(psi + nb[k]), acc);
      out[c] = fma(-T.nu, acc, out[c]);
    }
  }
}

// ---------------------------------------------------------------------------
// Bounded grid-wide barrier for co-resident (cooperatively launched) blocks.
// One arrival counter per barrier object: every block adds 1 except block 0,
// which adds 2^31 - (n - 1), so the n-th arrival flips bit 31 whatever the
// order and the low bits return to their value; a block waits for bit 31 to
// differ from what its own arrival saw (no separate release store).  Every
// wait gives up after kWaitNs of global time, records the timeout in *abort
// and returns false; a set abort word also ends every wait.
// ---------------------------------------------------------------------------
struct GridSync {
  unsigned int count;  // arrival counter (bit 31 flips once per barrier)
  int pad0[31];        // count alone on its 128-byte line
  unsigned int rgen;   // results published by grid reductions (incremented per reduction)
  int pad1[31];
  int abort;           // 0, or the SWE_ERR_* code that ended the launch
  int pad2[31];
};

constexpr unsigned long long kWaitNs = 4000000000ull;  // 4 s

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

// Arrival (thread 0 of block gb of gn co-resident blocks).  The fence
// publishes every write the block made before the caller's __syncthreads.
// Returns the value the counter had before this arrival; the arrival is the
// last one when it flipped bit 31.
__device__ __forceinline__ unsigned int flip_arrive(GridSync* s, int gb, int gn, bool* last) {
  const unsigned int add = gb == 0 ? 0x80000000u - (unsigned int)(gn - 1) : 1u;
  __threadfence();
  const unsigned int old = atomicAdd(&s->count, add);
  *last = ((old ^ (old + add)) & 0x80000000u) != 0;
  return old;
}

// Bounded spin until cond() is false; checks the abort word and the time
// limit (kWaitNs unless given) every 64 polls.  Returns false on abort or
// timeout.
template <class Cond>
__device__ __forceinline__ bool bounded_spin(GridSync* s, int timeout_code, Cond cond,
                                             unsigned long long limit_ns = kWaitNs) {
  unsigned long long t0 = 0;
  for (unsigned int it = 0; cond(); ++it) {
    if ((it & 63u) == 63u) {
      if (ld_volatile_int(&s->abort) != 0) return false;
      const unsigned long long now = globaltimer();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > limit_ns) {
        atomicCAS(&s->abort, 0, timeout_code);
        return false;
      }
      if (it > 4096u) __nanosleep(128);  // a long wait: back off
    }
  }
  return true;
}

// Thread 0 of block gb: arrive and wait for all gn blocks.  The caller
// separates the block's threads with __syncthreads on both sides; the fence
// after the wait makes every block's earlier writes visible to this block.
__device__ __forceinline__ bool flip_barrier(GridSync* s, int gb, int gn, int timeout_code) {
  bool last;
  const unsigned int old = flip_arrive(s, gb, gn, &last);
  if (!last) {
    const volatile unsigned int* c = &s->count;
    if (!bounded_spin(s, timeout_code, [&] { return ((old ^ *c) & 0x80000000u) == 0; })) return false;
  }
  __threadfence();
  return ld_volatile_int(&s->abort) == 0;
}

}  // namespace swe
