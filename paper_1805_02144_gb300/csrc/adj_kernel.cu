// Adjoint of one phipm_simul_iom2 evaluation (Sec. 4.3, Algorithm 1) with the
// substep decisions frozen, as one persistent cooperative launch.
//
// The forward launch, run in tape mode, kept for every accepted substep k its
// w_0..w_p (Eq. eq3.18), its raw IOM2 basis and the scalars of the substep
// (t_k, tau_k, beta, H_m, basis scales, scaling steps of the exponential).
// This launch walks the substeps backwards.  For substep k, with Y the
// adjoint of y_{k+1}:
//   1. update (Eq. eq3.17, corrected Krylov formula): adjoints of w_j (j < p),
//      of the basis vectors (alpha_r Y), of phi_p(tau H) e_1, of the last entry
//      of phi_{p+1}(tau H) e_1, of h_{m+1,m} and of beta, from the m+1 dots
//      <v_r, Y> (one wide grid reduction);
//   2. the augmented exponential: the reverse of the scaled Taylor evaluation
//      the forward used (same polynomial, same scaling), giving the adjoint of
//      the tridiagonal H_m (last block of the reduction, whole block);
//   3. IOM2, column j = m-1 .. 0 (z = A v_j, two window dots, norm): with
//      zbar' = Vbar_{j+1}/eta + etabar v_{j+1} and zbar = zbar' + abar v_{j-1}
//      + bbar v_j, the column adds A^T zbar - b zbar' + bbar z to Vbar_j,
//      -a zbar' + abar z to Vbar_{j-1}, and dt Q'(v_j)^T zbar to the
//      linearisation state's adjoint (A = dt J(u), J(u) = J(0) + Q'(u)).
//      Two phases per column, like the forward: (B) zbar and the transposed
//      pass-1 planes, neighbours' zbar rebuilt from the four vectors it is
//      made of so that no barrier separates forming and gathering it; (C) the
//      fused J^T / Q'^T pass 2, the updates and the next column's five dots;
//   4. beta = ||w_p||, v_0 = w_p / beta, then the w_j recurrence backwards
//      (A^T and Q'^T of w_{j-1} for every product that was not skipped), which
//      ends with the adjoint of y_k.
// Reductions are summed in a fixed order (bitwise reproducible per grid size);
// every wait is bounded (the forward kernel's grid barrier).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/swe_exprb.h"
#include "adj_args.h"
#include "grid_ops.cuh"
#include "phi_args.h"
#include "swe_dev.cuh"

namespace swe {

constexpr int ADJ_THREADS = 384;
constexpr int ADJ_MINB = 1;
constexpr int ADJ_TAYLOR_TERMS = 32;  // the forward's Taylor degree
constexpr int MW = KMAX + PMAX + 2;   // rows of the augmented matrix (max)

// Coefficients of one IOM2 column's reverse (computed per block by thread 0).
struct ColCoef {
  double kv, kr1, krm, krj;  // zbar  = kv Vb1 + kr1 r_{j+1} + krm r_{j-1} + krj r_j
  double pv, pr1;            // zbar' = pv Vb1 + pr1 r_{j+1}
  double zr1, zrm, zrj;      // z     = zr1 r_{j+1} + zrm r_{j-1} + zrj r_j
  double xa, xb, xy, xp;     // Vbar_j = xy Y + xp P_j + xa zbar' + xb z + dt J^T zbar
  double pa, pb;             // P_{j-1} = pa zbar' + pb z
  double vx, vy;             // Vb1 = vx X_{j+1} + vy Y
  double sj;                 // v_j = sj r_j
};

struct AdjShared {
  int gb, gn;
  unsigned long long t_last;
  double red[(ADJ_THREADS / 32) * NRED];
  int ok;
  ColCoef cc;
  double ck[ADJ_TAYLOR_TERMS + 2];
  double tb[MW + 2], ob[MW + 2], xv[MW + 2];
  double hd[KMAX + 1], hu[KMAX + 1], hl[KMAX + 2];
  double scal[8];
};

enum AdjPhase { AP_A = 0, AP_B, AP_C, AP_WB, AP_WC };

// ---------------------------------------------------------------------------
// Transposed stencil pieces on a vector lam (rebuilt on the fly at any cell by
// `lamf(cell, comp)`), for J(u)^T with aux = (eta, P) of u and Q'(x)^T.
// ---------------------------------------------------------------------------

// Pass 1 at cell i.  Planes: 0 a_n = P(u).lam_u, 1 a_x = (n x x_u).lam_u,
// 2..4 P_n lam_u, 5..8 L^T lam, 9 V.x_u (relative vorticity of x).  Also
// writes lam itself (4 planes of Zb).
template <class LamF>
__device__ __forceinline__ void adj_pass1(const Tables& T, int i, LamF lamf, const double* aux, const double* x,
                                          double* PL, double* Zb) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, i, nb);
  double lu[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    lu[c] = lamf(i, c);
    Zb[(size_t)c * ng + i] = lu[c];
  }
  const double n0 = ldtab(T.nrm + i), n1 = ldtab(T.nrm + ng + i), n2 = ldtab(T.nrm + 2 * (size_t)ng + i);
  const double p0 = ld(aux + (size_t)ng + i), p1 = ld(aux + 2 * (size_t)ng + i), p2 = ld(aux + 3 * (size_t)ng + i);
  PL[i] = fma(p0, lu[0], fma(p1, lu[1], p2 * lu[2]));
  const double x0 = ld(x + i), x1 = ld(x + (size_t)ng + i), x2 = ld(x + 2 * (size_t)ng + i);
  const double q0 = n1 * x2 - n2 * x1, q1 = n2 * x0 - n0 * x2, q2 = n0 * x1 - n1 * x0;
  PL[(size_t)ng + i] = fma(q0, lu[0], fma(q1, lu[1], q2 * lu[2]));
  const double nl = fma(n0, lu[0], fma(n1, lu[1], n2 * lu[2]));
  PL[2 * (size_t)ng + i] = fma(-n0, nl, lu[0]);
  PL[3 * (size_t)ng + i] = fma(-n1, nl, lu[1]);
  PL[4 * (size_t)ng + i] = fma(-n2, nl, lu[2]);
  double lt[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) lt[c] = ldtab(T.wld + i) * lu[c];
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    const double w = ldtab(T.wlT + (size_t)k * ng + i);
#pragma unroll
    for (int c = 0; c < 4; ++c) lt[c] = fma(w, lamf(nb[k], c), lt[c]);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) PL[(size_t)(5 + c) * ng + i] = lt[c];
  double vor = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) vor = fma(ldtab(T.vd + (size_t)c * ng + i), ld(x + (size_t)c * ng + i), vor);
#pragma unroll
  for (int k = 0; k < SLOTS; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      vor = fma(ldtab(T.vc + ((size_t)c * SLOTS + k) * ng + i), ld(x + (size_t)c * ng + nb[k]), vor);
  PL[9 * (size_t)ng + i] = vor;
}

// Pass 2 at cell j: jt = J(u)^T lam, qt = Q'(x)^T lam from the pass-1 planes.
__device__ __forceinline__ void adj_pass2(const Tables& T, int j, const double* u, const double* aux,
                                          const double* x, const double* PL, const double* Zb, double jt[4],
                                          double qt[4]) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, j, nb);
  const double* An = PL;
  const double* Ax = PL + (size_t)ng;
  const double* Bp = PL + 2 * (size_t)ng;
  const double* Lt = PL + 5 * (size_t)ng;
  const double* Zh = Zb + 3 * (size_t)ng;
  double van[3], vax[3], qb[3], sb = 0.0, ll[4];
  {
    const double an = ld(An + j), ax = ld(Ax + j), zh = ld(Zh + j);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double vd = ldtab(T.vd + (size_t)c * ng + j);
      van[c] = vd * an;
      vax[c] = vd * ax;
      sb = fma(ldtab(T.gdg + (size_t)c * ng + j), ld(Bp + (size_t)c * ng + j), sb);
      qb[c] = ldtab(T.ndd + (size_t)c * ng + j) * zh;
    }
    const double wd = ldtab(T.wld + j);
#pragma unroll
    for (int c = 0; c < 4; ++c) ll[c] = wd * ld(Lt + (size_t)c * ng + j);
  }
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    const int i = nb[k];
    const double an = ld(An + i), ax = ld(Ax + i), zh = ld(Zh + i);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double wv = ldtab(T.vcT + ((size_t)c * SLOTS + k) * ng + j);
      const double wn = ldtab(T.ncT + ((size_t)c * SLOTS + k) * ng + j);
      van[c] = fma(wv, an, van[c]);
      vax[c] = fma(wv, ax, vax[c]);
      sb = fma(wn, ld(Bp + (size_t)c * ng + i), sb);
      qb[c] = fma(wn, zh, qb[c]);
    }
    const double wl = ldtab(T.wlT + (size_t)k * ng + j);
#pragma unroll
    for (int c = 0; c < 4; ++c) ll[c] = fma(wl, ld(Lt + (size_t)c * ng + i), ll[c]);
  }
  sb = -sb;
  const double n0 = ldtab(T.nrm + j), n1 = ldtab(T.nrm + ng + j), n2 = ldtab(T.nrm + 2 * (size_t)ng + j);
  const double l0 = ld(Zb + j), l1 = ld(Zb + (size_t)ng + j), l2 = ld(Zb + 2 * (size_t)ng + j);
  const double c0 = n1 * l2 - n2 * l1, c1 = n2 * l0 - n0 * l2, c2 = n0 * l1 - n1 * l0;  // n x lam_u
  const double eta_n = ld(aux + j), eta_x = ld(PL + 9 * (size_t)ng + j);
  double uv[4], xv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uv[c] = ld(u + (size_t)c * ng + j);
    xv[c] = ld(x + (size_t)c * ng + j);
  }
  const double cr[3] = {c0, c1, c2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    jt[c] = fma(uv[c], sb, fma(-uv[3], qb[c], fma(eta_n, cr[c], -van[c])));
    qt[c] = fma(xv[c], sb, fma(-xv[3], qb[c], fma(eta_x, cr[c], -vax[c])));
  }
  jt[3] = fma(T.g, sb, -fma(uv[0], qb[0], fma(uv[1], qb[1], uv[2] * qb[2])));
  qt[3] = -fma(xv[0], qb[0], fma(xv[1], qb[1], xv[2] * qb[2]));
  // transposed dissipation -nu L^T L^T lam on every variable (J only)
#pragma unroll
  for (int c = 0; c < 4; ++c) jt[c] = fma(-T.nu, ll[c], jt[c]);
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// Raw basis slot j of substep k (slot 0 is w_p).
__device__ __forceinline__ const double* raw_vec(const AdjArgs& a, int k, int j) {
  const size_t n = (size_t)4 * a.T.ng;
  if (j == 0) return a.tapeW + (size_t)k * (a.p + 1) * n + (size_t)a.p * n;
  return a.tapeV + a.tape_offV[k] + (size_t)j * n;
}

template <class SH>
__device__ __forceinline__ void adj_abort(const AdjArgs& a, SH& sh, int code) {
  if (threadIdx.x == 0) {
    a.ctrl->status = code;
    atomicCAS(&a.sync->abort, 0, code);
  }
  (void)sh;
}

// Wide grid reduction: nv dot products <vecs_r, Y> over all cells (vecs_r for
// r < nv0: raw basis slots of substep k; r = nv0, nv0+1: <r_m, r_{m-2}>,
// <r_m, r_{m-1}>), summed per block in a fixed order, then over blocks in a
// fixed order (sum_strided) by block 0, which runs `last()` with all its
// threads between two grid barriers.
template <class LastFn>
__device__ bool adj_wide_reduce(const AdjArgs& a, AdjShared& sh, const CellLoop& CL, int k, const TapeSub& S,
                                int m, LastFn last) {
  const int ng = a.T.ng;
  const int nv = m + 3;
  for (int r = 0; r < nv; ++r) {
    const double* x;
    const double* y;
    if (r <= m) {
      x = raw_vec(a, k, r);
      y = a.Y;
    } else {
      x = raw_vec(a, k, m);
      const int jj = r == m + 1 ? m - 2 : m - 1;
      y = jj >= 0 ? raw_vec(a, k, jj) : nullptr;
    }
    double acc = 0.0;
    if (y)
      FOR_CELLS(i)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const size_t e = (size_t)c * ng + i;
          acc = fma(ld(x + e), ld(y + e), acc);
        }
    double v1[1] = {acc};
    block_sum<1>(v1, sh.red);
    if (threadIdx.x == 0) a.partw[(size_t)sh.gb * ADJ_KW + r] = v1[0];
  }
  // all block totals published; block 0 sums them in a fixed order and runs
  // `last` with all its threads while the others wait at the second barrier
  if (!grid_barrier(a, sh, AP_A)) return false;
  if (sh.gb == 0) {
    for (int r = threadIdx.x; r < nv; r += blockDim.x) {
      a.ctrl->wide[r] = sum_strided(a.partw + r, ADJ_KW, sh.gn);
    }
    __syncthreads();
    last();
    __syncthreads();
  }
  return grid_barrier(a, sh, AP_A);
}

// Row r < m of tau H times v (the forward's operation order).
__device__ __forceinline__ double h_row(const AdjShared& sh, int r, int m, double tau, const double* v) {
  double s = tau * sh.hd[r] * v[r];
  if (r > 0) s = fma(tau * sh.hl[r], v[r - 1], s);
  if (r < m - 1) s = fma(tau * sh.hu[r], v[r + 1], s);
  return s;
}

// Row r of the augmented matrix X times v: tau H in the first m rows plus
// X[0][m] = 1, and X[r][r+1] = 1 for m <= r < m+p.
__device__ __forceinline__ double aug_row(const AdjShared& sh, int r, int m, int p, double tau,
                                          const double* v) {
  if (r < m) {
    double s = h_row(sh, r, m, tau, v);
    if (r == 0) s += v[m];
    return s;
  }
  if (r < m + p) return v[r + 1];
  return 0.0;
}

// Column q of X^T v: sum_r X[r][q] v[r].
__device__ __forceinline__ double aug_col(const AdjShared& sh, int q, int m, double tau, const double* v) {
  if (q < m) {
    double s = tau * sh.hd[q] * v[q];
    if (q > 0) s = fma(tau * sh.hu[q - 1], v[q - 1], s);
    if (q < m - 1) s = fma(tau * sh.hl[q + 1], v[q + 1], s);
    return s;
  }
  if (q == m) return v[0];
  return v[q - 1];
}

// Steps 1 and 2 for substep k (all threads of the block that summed the wide
// reduction).  ctrl->wide holds raw dots <r_r, Y> (r <= m) and the two basis
// dots.  Writes alpha_r, the H adjoints, betabar and the first column's
// scalars.
__device__ void adj_exp_reverse(const AdjArgs& a, AdjShared& sh, const TapeSub& S) {
  AdjCtrl* C = a.ctrl;
  const int r = threadIdx.x;
  const int m = S.m, p = a.p, M = m + p + 1;
  const double tau = S.tau, beta = S.beta, h = S.hnext;
  const int s = S.s;
  double* xs = a.xs;                           // s x MW: x at the start of each scaling step
  double* ts = a.xs + (size_t)a.xs_steps * MW;  // (TERMS+1) x MW: Taylor terms of one step
  for (int q = r; q <= m; q += blockDim.x) {
    sh.hd[q] = S.hd[q];
    sh.hu[q] = S.hu[q];
    sh.hl[q] = S.hl[q];
  }
  if (r >= 1 && r <= ADJ_TAYLOR_TERMS) sh.ck[r] = 1.0 / ((double)s * (double)r);
  if (r < M) sh.xv[r] = (r == M - 1) ? 1.0 : 0.0;
  __syncthreads();
  // forward: x = (T_32(X/s))^s e_{M-1}, keeping the start of each step; the
  // terms alternate between sh.xv and sh.ob (one block barrier per term)
  {
    double* buf[2] = {sh.xv, sh.ob};
    int c = 0;
    for (int st = 0; st < s; ++st) {
      double acc = r < M ? buf[c][r] : 0.0;
      if (r < M) xs[(size_t)st * MW + r] = acc;
      for (int kk = 1; kk <= ADJ_TAYLOR_TERMS; ++kk) {
        const double v = r < M ? sh.ck[kk] * aug_row(sh, r, m, p, tau, buf[c]) : 0.0;
        if (r < M) {
          buf[c ^ 1][r] = v;
          acc += v;
        }
        __syncthreads();
        c ^= 1;
      }
      if (r < M) buf[c ^ 1][r] = acc;
      __syncthreads();
      c ^= 1;
    }
    if (c != 0) {
      const double v = r < M ? buf[c][r] : 0.0;
      __syncthreads();
      if (r < M) sh.xv[r] = v;
      __syncthreads();
    }
  }
  // phi_{p+1}(tau H) e_1 = x[0:m]; phi_p(tau H) e_1 = tau H x + e_1 / p!
  double fact = 1.0;
  for (int q = 2; q <= p; ++q) fact *= q;
  const double tp = pow(tau, (double)p);
  double yr = 0.0, g_r = 0.0;
  if (r < m) {
    yr = h_row(sh, r, m, tau, sh.xv);
    if (r == 0) yr += 1.0 / fact;
    g_r = S.sig[r] * ((volatile double*)C->wide)[r];
  }
  const double xm1 = sh.xv[m - 1];
  const double g_m = S.sig[m] * ((volatile double*)C->wide)[m];
  // combine coefficients of the normalised basis and the adjoints of the
  // exponential's outputs
  if (r < m) C->alpha[r] = tp * beta * yr;
  if (r == 0) C->alpha[m] = tp * beta * tau * h * xm1;
  // ob = adjoint of phi_p e_1 (cbar), tb = adjoint of x
  if (r < m) sh.ob[r] = tp * beta * g_r;
  __syncthreads();
  // beta-bar (fixed order, thread 0)
  if (r == 0) {
    double bb = 0.0;
    for (int q = 0; q < m; ++q) {
      double yq = h_row(sh, q, m, tau, sh.xv);
      if (q == 0) yq += 1.0 / fact;
      bb = fma(yq, S.sig[q] * ((volatile double*)C->wide)[q], bb);
    }
    C->betabar = tp * (bb + tau * h * xm1 * g_m);
    C->hlb[m] = tp * beta * tau * xm1 * g_m;
  }
  // xbar = (tau H)^T cbar (first m rows), + dbar at m-1
  double xb = 0.0;
  if (r < m) {
    double s2 = tau * sh.hd[r] * sh.ob[r];
    if (r > 0) s2 = fma(tau * sh.hu[r - 1], sh.ob[r - 1], s2);
    if (r < m - 1) s2 = fma(tau * sh.hl[r + 1], sh.ob[r + 1], s2);
    xb = s2;
  }
  if (r == m - 1) xb += tp * beta * tau * h * g_m;
  // Xbar band of row r (entries r-1, r, r+1) from phi_p = tau H x[0:m]
  double bl = 0.0, bd = 0.0, bu = 0.0;
  if (r < m) {
    bd = sh.ob[r] * sh.xv[r];
    if (r > 0) bl = sh.ob[r] * sh.xv[r - 1];
    if (r < m - 1) bu = sh.ob[r] * sh.xv[r + 1];
  }
  __syncthreads();
  if (r < M) sh.tb[r] = xb;
  __syncthreads();
  // reverse the scaling steps
  for (int st = s - 1; st >= 0; --st) {
    // recompute this step's Taylor terms into ts (each term is its own row,
    // so one block barrier per term suffices)
    if (r < M) ts[r] = xs[(size_t)st * MW + r];
    __syncthreads();
    for (int kk = 1; kk <= ADJ_TAYLOR_TERMS; ++kk) {
      const double v = r < M ? sh.ck[kk] * aug_row(sh, r, m, p, tau, ts + (size_t)(kk - 1) * MW) : 0.0;
      if (r < M) ts[(size_t)kk * MW + r] = v;
      __syncthreads();
    }
    // out = sum_k t_k; tbar_k = obar + ck[k+1] X^T tbar_{k+1}
    if (r < M) sh.ob[r] = sh.tb[r];  // obar
    __syncthreads();
    for (int kk = ADJ_TAYLOR_TERMS; kk >= 1; --kk) {
      // band of Xbar += ck tbar_k[r] t_{k-1}[q]
      if (r < m) {
        const double* tprev = ts + (size_t)(kk - 1) * MW;
        const double f = sh.ck[kk] * sh.tb[r];
        bd = fma(f, tprev[r], bd);
        if (r > 0) bl = fma(f, tprev[r - 1], bl);
        if (r < m - 1) bu = fma(f, tprev[r + 1], bu);
      }
      double v = r < M ? fma(sh.ck[kk], aug_col(sh, r, m, tau, sh.tb), sh.ob[r]) : 0.0;
      __syncthreads();
      if (r < M) sh.tb[r] = v;
      __syncthreads();
    }
  }
  // H adjoints (X = tau H)
  if (r < m) {
    C->hdb[r] = tau * bd;
    if (r > 0) C->hlb[r] = tau * bl;
    if (r < m - 1) C->hub[r] = tau * bu;
  }
  __syncthreads();
}

// Scalars of column j's reverse from its five dots (normalised vectors):
// D1 = <Vb_{j+1}, v_{j+1}>, D2 = <Vb_{j+1}, v_{j-1}>, D3 = <v_{j+1}, v_{j-1}>,
// D4 = <Vb_{j+1}, v_j>, D5 = <v_{j+1}, v_j>.  Thread 0.
__device__ void adj_column_scalars(volatile AdjCtrl* C, const TapeSub& S, int j, double D1, double D2,
                                   double D3, double D4, double D5) {
  const double eta = S.hl[j + 1];
  const double etab = C->hlb[j + 1] - D1 / eta;
  const double abar = j > 0 ? C->hub[j - 1] - (D2 / eta + etab * D3) : 0.0;
  const double bbar = C->hdb[j] - (D4 / eta + etab * D5);
  C->col[0] = etab;
  C->col[1] = abar;
  C->col[2] = bbar;
}

__device__ void load_colcoef(const AdjArgs& a, AdjShared& sh, const TapeSub& S, int j) {
  if (threadIdx.x == 0) {
    const AdjCtrl* C = a.ctrl;
    const int m = S.m;
    const double eta = S.hl[j + 1];
    const double etab = ((volatile const double*)C->col)[0];
    const double abar = ((volatile const double*)C->col)[1];
    const double bbar = ((volatile const double*)C->col)[2];
    const double s1 = S.sig[j + 1], sj = S.sig[j], sm = j > 0 ? S.sig[j - 1] : 0.0;
    const double av = j > 0 ? S.hu[j - 1] : 0.0, bv = S.hd[j];
    ColCoef& c = sh.cc;
    c.kv = 1.0 / eta;
    c.kr1 = etab * s1;
    c.krm = abar * sm;
    c.krj = bbar * sj;
    c.pv = 1.0 / eta;
    c.pr1 = etab * s1;
    c.zr1 = eta * s1;
    c.zrm = av * sm;
    c.zrj = bv * sj;
    c.xa = -bv;
    c.xb = bbar;
    c.xy = ((volatile const double*)C->alpha)[j];
    c.xp = (j == m - 1) ? 0.0 : 1.0;
    c.pa = -av;
    c.pb = abar;
    if (j == m - 1) {
      c.vx = 0.0;
      c.vy = ((volatile const double*)C->alpha)[m];
    } else {
      c.vx = 1.0;
      c.vy = 0.0;
    }
    c.sj = sj;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// the launch
// ---------------------------------------------------------------------------
__device__ bool adj_run(const AdjArgs& a, AdjShared& sh) {
  const Tables& T = a.T;
  const int ng = T.ng;
  const size_t n = (size_t)4 * ng;
  const int p = a.p;
  const int chunk = (ng + sh.gn - 1) / sh.gn;
  const Range RG{min(ng, sh.gb * chunk), min(ng, (sh.gb + 1) * chunk)};
  const CellLoop CL(RG);
  AdjCtrl* C = a.ctrl;
  double* Wb = a.Wb;  // (p+1) x n: adjoints of w_j
  if (threadIdx.x == 0) sh.t_last = globaltimer();

  for (int k = a.nsub - 1; k >= 0; --k) {
    const TapeSub& S = a.tape_sub[k];
    const int m = S.m;
    const bool kry = S.beta > 0.0;
    // the tape's scalars index buffers: check them against what the host laid out
    if ((kry && (S.broken || m < 1 || m > KMAX || m > a.tape_mmax[k] || S.s < 1 || S.s > a.xs_steps)) ||
        (S.land && (S.out_idx < 0 || S.out_idx >= a.ns))) {
      adj_abort(a, sh, SWE_ERR_INVALID_ARG);
      return false;
    }
    const double* yb = (S.land && a.ybar[S.out_idx]) ? a.ybar[S.out_idx] : nullptr;
    const bool first = (k == a.nsub - 1);
    // ---- phase A: Y, wbar_j = tau^j/j! Y (j < p), dots <r_r, Y> ------------
    double cw[PMAX + 1];
    {
      double f = 1.0, tpw = 1.0;
      for (int j = 0; j < p; ++j) {
        if (j > 0) {
          f *= (double)j;
          tpw *= S.tau;
        }
        cw[j] = tpw / f;
      }
    }
    FOR_CELLS(i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const size_t e = (size_t)c * ng + i;
        double y = first ? 0.0 : Wb[e];
        if (yb) y += ld(yb + e);
        a.Y[e] = y;
        for (int j = 0; j < p; ++j) Wb[(size_t)j * n + e] = cw[j] * y;
      }
    if (kry) {
      auto last = [&]() {
        adj_exp_reverse(a, sh, S);
        if (threadIdx.x == 0) {
          // first column (j = m-1): Vbar_m = alpha_m Y
          volatile AdjCtrl* VC = C;
          const double am = VC->alpha[m];
          const double gm = S.sig[m] * VC->wide[m];
          const double gm1 = S.sig[m - 1] * VC->wide[m - 1];
          const double gm2 = m >= 2 ? S.sig[m - 2] * VC->wide[m - 2] : 0.0;
          const double D3 = m >= 2 ? S.sig[m] * S.sig[m - 2] * VC->wide[m + 1] : 0.0;
          const double D5 = S.sig[m] * S.sig[m - 1] * VC->wide[m + 2];
          adj_column_scalars(VC, S, m - 1, am * gm, am * gm2, D3, am * gm1, D5);
        }
      };
      if (!adj_wide_reduce(a, sh, CL, k, S, m, last)) return false;

      // ---- IOM2 columns backwards ------------------------------------------
      for (int j = m - 1; j >= 0; --j) {
        load_colcoef(a, sh, S, j);
        const ColCoef cc = sh.cc;
        const double* r1 = raw_vec(a, k, j + 1);
        const double* rj = raw_vec(a, k, j);
        const double* rm = j > 0 ? raw_vec(a, k, j - 1) : nullptr;
        const double* X1 = a.X + (size_t)((j + 1) & 1) * n;
        double* Xj = a.X + (size_t)(j & 1) * n;
        const double* Pj = a.P + (size_t)(j & 1) * n;
        double* Pm = a.P + (size_t)((j + 1) & 1) * n;  // P_{j-1}
        const double* Y = a.Y;
        auto vb1 = [&](size_t e) {
          double v = cc.vy * ld(Y + e);
          if (cc.vx != 0.0) v = fma(cc.vx, ld(X1 + e), v);
          return v;
        };
        auto zbar = [&](int cell, int c) {
          const size_t e = (size_t)c * ng + cell;
          double z = fma(cc.kv, vb1(e), cc.kr1 * ld(r1 + e));
          if (rm) z = fma(cc.krm, ld(rm + e), z);
          return fma(cc.krj, ld(rj + e), z);
        };
        // phase B
        FOR_CELLS(i) adj_pass1(T, i, zbar, a.aux, rj, a.PL, a.Zb);
        if (!grid_barrier(a, sh, AP_B)) return false;
        // phase C
        double d[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        const double* rj2 = j >= 2 ? raw_vec(a, k, j - 2) : nullptr;
        const double dtsj = a.dt * cc.sj;
        FOR_CELLS(i) {
          double jt[4], qt[4];
          adj_pass2(T, i, a.u_lin, a.aux, rj, a.PL, a.Zb, jt, qt);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const size_t e = (size_t)c * ng + i;
            const double vv = vb1(e), v1 = ld(r1 + e), vj = ld(rj + e);
            const double vm = rm ? ld(rm + e) : 0.0;
            const double zp = fma(cc.pv, vv, cc.pr1 * v1);
            const double z = fma(cc.zr1, v1, fma(cc.zrm, vm, cc.zrj * vj));
            double x = fma(cc.xy, ld(Y + e), fma(cc.xa, zp, fma(cc.xb, z, a.dt * jt[c])));
            if (cc.xp != 0.0) x += ld(Pj + e);
            Xj[e] = x;
            if (rm) Pm[e] = fma(cc.pa, zp, cc.pb * z);
            a.ubar[e] = fma(dtsj, qt[c], a.ubar[e]);
            d[0] = fma(x, vj, d[0]);
            if (rj2) {
              const double v2 = ld(rj2 + e);
              d[1] = fma(x, v2, d[1]);
              d[2] = fma(vj, v2, d[2]);
            }
            if (rm) {
              d[3] = fma(x, vm, d[3]);
              d[4] = fma(vj, vm, d[4]);
            }
          }
        }
        const TapeSub* Sp = &S;
        auto post = [Sp, j](volatile AdjCtrl* c, bool, const auto& r) {
          volatile AdjCtrl* cc2 = c;
          const TapeSub& St = *Sp;
          if (j >= 1) {
            const int jn = j - 1;  // next column: Vb_{jn+1} = Vbar_j
            const double sj = St.sig[j], sm = St.sig[j - 1], s2 = j >= 2 ? St.sig[j - 2] : 0.0;
            adj_column_scalars(cc2, St, jn, sj * r[0], s2 * r[1], sj * s2 * r[2], sm * r[3], sj * sm * r[4]);
          } else {
            cc2->col[3] = St.sig[0] * r[0];  // <Vbar_0, v_0>
          }
        };
        if (!grid_reduce<5>(a, sh, d, AP_C, post)) return false;
      }
    }
    // ---- beta, v_0 = w_p / beta, then the w_j recurrence backwards ---------
    double wx = 0.0, wr = 0.0;
    if (kry) {
      const double D0 = ((volatile const double*)C->col)[3];
      const double bb = ((volatile const double*)&C->betabar)[0];
      wx = 1.0 / S.beta;
      wr = (bb - D0 / S.beta) * S.sig[0];
    }
    const double* X0 = a.X;
    const double* r0 = raw_vec(a, k, 0);
    const double* Wk = a.tapeW + (size_t)k * (p + 1) * n;
    for (int j = p; j >= 1; --j) {
      const bool nz = S.wnz[j - 1] != 0;
      auto lam = [&](int cell, int c) {
        const size_t e = (size_t)c * ng + cell;
        if (j == p) return kry ? fma(wx, ld(X0 + e), wr * ld(r0 + e)) : 0.0;
        return ld(Wb + (size_t)j * n + e);
      };
      double cl[PMAX + 1];
      {
        double f = 1.0, tpw = 1.0;
        for (int l = 0; l <= p - j; ++l) {
          if (l > 0) {
            f *= (double)l;
            tpw *= S.t;
          }
          cl[l] = tpw / f;
        }
      }
      const double* wprev = Wk + (size_t)(j - 1) * n;
      FOR_CELLS(i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const size_t e = (size_t)c * ng + i;
          const double lv = lam(i, c);
          for (int l = 0; l <= p - j; ++l)
            if (a.vbar[j + l]) a.vbar[j + l][e] = fma(cl[l], lv, a.vbar[j + l][e]);
        }
        if (nz) adj_pass1(T, i, lam, a.aux, wprev, a.PL, a.Zb);
      }
      if (nz) {
        if (!grid_barrier(a, sh, AP_WB)) return false;
        FOR_CELLS(i) {
          double jt[4], qt[4];
          adj_pass2(T, i, a.u_lin, a.aux, wprev, a.PL, a.Zb, jt, qt);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const size_t e = (size_t)c * ng + i;
            Wb[(size_t)(j - 1) * n + e] = fma(a.dt, jt[c], Wb[(size_t)(j - 1) * n + e]);
            a.ubar[e] = fma(a.dt, qt[c], a.ubar[e]);
          }
        }
      }
      if (!grid_barrier(a, sh, AP_WC)) return false;
    }
  }
  // y_0 = v_0
  if (a.nsub > 0 && a.vbar[0])
    FOR_CELLS(i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const size_t e = (size_t)c * ng + i;
        a.vbar[0][e] += Wb[e];
      }
  return true;
}

__global__ void __launch_bounds__(ADJ_THREADS, ADJ_MINB) adj_kernel(AdjArgs a) {
  __shared__ AdjShared sh;
  if (threadIdx.x == 0) {
    sh.gb = blockIdx.x;
    sh.gn = gridDim.x;
  }
  __syncthreads();
  bool ok = adj_run(a, sh);
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) {
    int ab = ld_volatile_int(&a.sync->abort);
    if (a.ctrl->status == SWE_OK) a.ctrl->status = ab != 0 ? ab : SWE_ERR_TIMEOUT;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.status_out) {
    // other blocks may still be leaving after an abort; their statuses are the same
    const int st = ld_volatile_int(&a.ctrl->status);
    if (st != SWE_OK && *a.status_out == SWE_OK) *a.status_out = st;
  }
}

int adj_max_blocks(int* nblocks, int* threads) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, adj_kernel, ADJ_THREADS, 0) != cudaSuccess) return -1;
  if (per < 1) return -1;
  *nblocks = sms * per;
  *threads = ADJ_THREADS;
  return 0;
}

int launch_adj_kernel(const AdjArgs& a, int nblocks, cudaStream_t st) {
  void* args[] = {(void*)&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)adj_kernel, dim3(nblocks), dim3(ADJ_THREADS), args, 0, st);
  return (int)e;
}

}  // namespace swe
