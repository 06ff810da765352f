// phipm_simul_iom2 (Sec. 4.3, Algorithm 1) as one persistent, cooperatively
// launched kernel: the w_j recurrence (Eq. eq3.18), the IOM2 Krylov sweep
// (Algorithm 1 step 2(i)), the augmented exponential, error estimate and
// substep controller (steps 2(ii)-6) and the substep update (Eq. eq3.17) all
// run on the device; the host launches once per call.
//
// Work split: block b owns a contiguous range of cells (space-filling-curve
// order, so its stencil gathers stay mostly inside the range).  Phases are
// separated by bounded grid barriers; reductions are summed per block as a
// fixed tree, then over blocks as a fixed tree by the last block to arrive,
// so results are bitwise reproducible for a given grid and launch shape.
// The small decisions (exponential of the (m+p+1)-square augmented matrix,
// controller) run on block 0 while the other blocks wait at the barrier.
//
// The Krylov basis is stored unnormalised: raw slot j holds z_j (slot 0 is
// w_p itself) and v_j = sig[j] * raw_j with sig[0] = 1/beta,
// sig[j+1] = 1/h_{j+1,j}; every use folds the scale into its coefficients.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/swe_exprb.h"
#include "grid_ops.cuh"
#include "phi_args.h"
#include "swe_dev.cuh"

namespace swe {

constexpr int PHI_MAX_THREADS = 512;  // largest block size of any instantiation (sizes Shared::red)
constexpr double TAYLOR_THETA = 4.0;
// Largest ||tau Hhat||_1 the scaled Taylor evaluation accepts (1024 scaling
// steps); beyond it (or when it is not finite) the call fails with NOCONV, as
// it only happens for states or step sizes that have already gone wrong.
constexpr double HNORM_MAX = 1024.0 * TAYLOR_THETA;

// Phase classes timed by block 0 while profiling: time from the end of the
// previous barrier to the end of this one (work plus wait).
enum Phase { PH_PROLOGUE = 0, PH_W_PASS1, PH_W_PASS2, PH_K_PASS1, PH_K_PASS2, PH_ORTH, PH_DECIDE, PH_COMBINE,
             PH_TAYLOR, PH_CONTROL };

struct Shared {
  int gb, gn;  // this block's index in its group of co-operating blocks, group size
  unsigned long long t_last;
  double red[(PHI_MAX_THREADS / 32) * NRED];
  double coef[KMAX + PMAX + 4];
  float coeff[KMAX + PMAX + 4];
  int ok;
  // decision scratch (block 0, warp 0)
  double x[KMAX + PMAX + 8], y[KMAX + PMAX + 8];
  double ck[40];
  double hd[KMAX + 1], hu[KMAX + 1], hl[KMAX + 2];
  double scal[4];
};


// Storage of the current substep: Wk holds w_0..w_p, Vk the raw basis slots
// j >= 1 (raw slot 0 is w_p itself).  Without a tape both are the fixed
// workspace; with a tape, substep k has its own regions.
template <typename R>
struct SubBufs {
  R* Wk;
  R* Vk;
  R* Wnext;  // where y_{k+1} goes
  __device__ __forceinline__ R* raw(int j, size_t n, int p) const {
    return j == 0 ? Wk + (size_t)p * n : Vk + (size_t)j * n;
  }
};

template <typename R>
__device__ __forceinline__ SubBufs<R> sub_bufs(const PhiArgsT<R>& a, int k) {
  const size_t n = (size_t)4 * a.T.ng;
  SubBufs<R> b;
  if (a.tapeW) {
    const size_t reg = (size_t)(a.p + 1) * n;
    b.Wk = a.tapeW + (size_t)k * reg;
    b.Vk = a.tapeV + a.tape_offV[k];
    b.Wnext = a.tapeW + (size_t)(k + 1) * reg;
  } else {
    b.Wk = a.W;
    b.Vk = a.Vbuf;
    b.Wnext = a.W;
  }
  return b;
}

__device__ __forceinline__ int taylor_steps(double hnorm) {
  return (int)fmax(1.0, ceil(hnorm / TAYLOR_THETA));
}

// ---------------------------------------------------------------------------
// Augmented exponential by scaled Taylor series (all threads of block 0, one
// row per thread).  Hhat (size M = m+p+1): Hhat[0:m,0:m] = tau H_m
// (tridiagonal), Hhat[0,m] = 1, Hhat[m+k, m+k+1] = 1 (k < p).  The last column
// of exp(Hhat) holds phi_{p+1}(tau H) e_1 in its first m rows:
// exp(Hhat) e_{M-1} = (exp(Hhat/s))^s e_{M-1}, s = ceil(||Hhat||_1 / THETA),
// each factor the Taylor polynomial of degree TAYLOR_TERMS.  With
// ||Hhat/s||_1 <= 4 the truncated tail is below 4^33/33! < 1e-17 of the
// vector, so a fixed degree needs no per-term convergence test.
// On return sh.x[0:m] = phi_{p+1}(tau H) e_1 and sh.y[0:m] = phi_p(tau H) e_1.
// ---------------------------------------------------------------------------
constexpr int TAYLOR_TERMS = 32;

// Entries of row r beyond the tridiagonal (iom > 2): sum over q = r+2 ..
// min(m-1, r+iom-1) of tau H[r][q] x[q], in ascending q (empty for IOM2).
__device__ __forceinline__ double hup_row(const double* hup, int iom, int r, int m, double tau, const double* x,
                                          double v) {
  const int qe = min(m - 1, r + iom - 1);
  for (int q = r + 2; q <= qe; ++q) v = fma(tau * __ldcg(hup + r * KMAX + q), x[q], v);
  return v;
}

__device__ void taylor_phi(Shared& sh, int m, int p, double tau, double hnorm, const double* hup, int iom) {
  const int r = threadIdx.x;
  const int M = m + p + 1;
  const int s = taylor_steps(hnorm);
  // row r of (tau H): coefficients held in registers
  double cd = 0.0, cl = 0.0, cu = 0.0;
  if (r < m) {
    cd = tau * sh.hd[r];
    if (r > 0) cl = tau * sh.hl[r];
    if (r < m - 1) cu = tau * sh.hu[r];
  }
  if (r >= 1 && r <= TAYLOR_TERMS) sh.ck[r] = 1.0 / ((double)s * (double)r);
  double acc = (r == M - 1) ? 1.0 : 0.0;
  if (r < M) sh.x[r] = acc;
  __syncthreads();
  // terms alternate between sh.x and sh.y: one barrier per term among the
  // warps that hold rows (named barrier 1, nact threads); the other warps of
  // the block wait at the block barrier below
  const int nact = ((M + 31) / 32) * 32;
  if (r < nact) {
    double* buf[2] = {sh.x, sh.y};
    int c = 0;
    for (int step = 0; step < s; ++step) {
      // buf[c] holds the current term (starting with the vector itself)
      for (int k = 1; k <= TAYLOR_TERMS; ++k) {
        const double* xc = buf[c];
        double v = 0.0;
        if (r < m) {
          v = cd * xc[r];
          if (r > 0) v = fma(cl, xc[r - 1], v);
          if (r < m - 1) v = fma(cu, xc[r + 1], v);
          if (iom > 2) v = hup_row(hup, iom, r, m, tau, xc, v);
          if (r == 0) v += xc[m];
          v *= sh.ck[k];
        } else if (r < m + p) {
          v = xc[r + 1] * sh.ck[k];
        }
        if (r < M) {
          buf[c ^ 1][r] = v;
          acc += v;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nact) : "memory");
        c ^= 1;
      }
      // the buffer read by the last term is free again: the step's sum goes there
      if (r < M) buf[c ^ 1][r] = acc;
      asm volatile("bar.sync 1, %0;" ::"r"(nact) : "memory");
      c ^= 1;
    }
    if (c != 0 && r < M) sh.x[r] = acc;  // leave x in sh.x
  }
  __syncthreads();
  // phi_p(tau H) e_1 = tau H phi_{p+1}(tau H) e_1 + e_1 / p!   (Eq. eq3.7)
  if (r < m) {
    double v = cd * sh.x[r];
    if (r > 0) v = fma(cl, sh.x[r - 1], v);
    if (r < m - 1) v = fma(cu, sh.x[r + 1], v);
    if (iom > 2) v = hup_row(hup, iom, r, m, tau, sh.x, v);
    if (r == 0) {
      double fact = 1.0;
      for (int k = 2; k <= p; ++k) fact *= k;
      v += 1.0 / fact;
    }
    sh.y[r] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ long long nint_d(double x) { return (long long)floor(x + 0.5); }

// C(tau, m) of Eq. eq:cost
__device__ double cost_fn(double tau, int m, int p, double remaining, double N, double nA,
                          double hnorm) {
  long long nsub = nint_d(remaining / tau);
  if (nsub < 1) nsub = 1;
  long long e = nint_d(log2(hnorm / 5.37));
  if (e < 0) e = 0;
  double M = 44.0 / 3.0 + 2.0 * (double)e;
  double mp = (double)(m + p + 1);
  return (double)nsub * (double)m * (N + nA) + 2.0 * (p - 1) * (nA + N) + M * mp * mp * mp +
         (2.0 * p + 1.0) * N;
}

// Error estimate, acceptance test and controller (Algorithm 1 steps 2(ii)-6),
// executed by all threads of block 0 (uniform control flow; the scalar
// controller runs on thread 0).  Writes the decision into ctrl.
template <class A>
__device__ void decide(const A& a, Shared& sh) {
  volatile PhiCtrl* C = a.ctrl;
  const int lane = threadIdx.x;
  const int p = a.p;
  const double t = C->t, t_out = C->t_out;
  const double remaining = t_out - t;
  const double beta = C->beta;
  double tau_nom;
  int m;
  int rec_acc = 0;
  const bool replay = a.replay != nullptr;
  if (replay) {
    int pos = C->replay_pos;
    if (pos >= a.n_replay) {
      if (lane == 0) {
        C->status = SWE_ERR_INVALID_ARG;
        abort_launch(a, SWE_ERR_INVALID_ARG);
      }
      return;
    }
    tau_nom = a.replay[3 * pos];
    m = (int)a.replay[3 * pos + 1];
    rec_acc = a.replay[3 * pos + 2] != 0.0;
  } else {
    tau_nom = C->tau;
    m = C->m;
  }
  const bool land = tau_nom >= remaining * (1.0 - 1e-12);
  const double tau_k = land ? remaining : tau_nom;

  int m_use = m;
  double eps = 0.0, hnorm = 1.0, hnext = 0.0;
  if (beta > 0.0) {
    m_use = min(m, (int)C->size);
    for (int r = lane; r <= m_use; r += blockDim.x) {
      sh.hd[r] = C->hd[r];
      sh.hu[r] = C->hu[r];
      sh.hl[r] = C->hl[r];
    }
    __syncthreads();
    if (lane < 32) {  // max column sum of |H_m| (max is exact in any order)
      double cs = 0.0;
      for (int j = lane; j < m_use; j += 32) {
        double s = fabs(sh.hd[j]);
        if (j > 0) s += fabs(sh.hu[j - 1]);
        if (j + 1 < m_use) s += fabs(sh.hl[j + 1]);
        if (a.iom > 2)
          for (int i = max(0, j - a.iom + 1); i <= j - 2; ++i)
            s += fabs(__ldcg((const double*)a.ctrl->hup + i * KMAX + j));
        cs = fmax(cs, s);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cs = fmax(cs, __shfl_xor_sync(0xffffffffu, cs, o));
      if (lane == 0) sh.scal[0] = cs;
    }
    __syncthreads();
    hnorm = fmax(tau_k * sh.scal[0], 1.0);
    if (!(hnorm <= HNORM_MAX)) {  // uniform in the block: every lane sees the same value
      if (lane == 0) {
        C->status = SWE_ERR_NOCONV;
        abort_launch(a, SWE_ERR_NOCONV);
      }
      return;
    }
    phase_tick(a, sh, PH_CONTROL);
    taylor_phi(sh, m_use, p, tau_k, hnorm, (const double*)a.ctrl->hup, a.iom);
    phase_tick(a, sh, PH_TAYLOR);
  }
  // The rest is scalar work: warp 0 alone, its lanes evaluating the powers and
  // the two costs side by side (the other warps wait at the next barrier).
  if (lane >= 32) return;
  constexpr unsigned FULL = 0xffffffffu;
  const double pw = pow(tau_k, (double)min(lane, p));  // lane j <= p: tau_k^j
  const double tp = __shfl_sync(FULL, pw, p);
  if (beta > 0.0) {
    hnext = (C->broken && m_use == C->size) ? 0.0 : sh.hl[m_use];
    eps = tp * beta * tau_k * fabs(hnext) * fabs(sh.x[m_use - 1]);
  }
  double tpow[PMAX];
#pragma unroll
  for (int j = 0; j < PMAX; ++j) tpow[j] = __shfl_sync(FULL, pw, min(j, p));
  const double omega = t_out * eps / (tau_k * a.tol * C->scale);
  const bool accepted = replay ? (rec_acc != 0) : (omega <= a.delta);

  // combination coefficients (warp 0, then lane 0 finishes the scalars)
  if (accepted) {
    if (beta > 0.0) {
      for (int r = lane; r < m_use; r += 32) C->cV[r] = tp * beta * sh.y[r] * C->sig[r];
      if (lane == 0)
        C->cV[m_use] = hnext != 0.0 ? tp * beta * tau_k * hnext * sh.x[m_use - 1] * C->sig[m_use] : 0.0;
    }
    if (a.tape_sub) {  // keep what the adjoint needs of this substep
      TapeSub& S = a.tape_sub[C->n_sub];
      if (beta > 0.0)
        for (int r = lane; r <= m_use; r += 32) {
          S.sig[r] = C->sig[r];
          S.hd[r] = sh.hd[r];
          S.hu[r] = sh.hu[r];
          S.hl[r] = sh.hl[r];
        }
      if (lane == 0) {
        S.t = t;
        S.tau = tau_k;
        S.beta = beta;
        S.hnext = hnext;
        S.m = m_use;
        S.s = beta > 0.0 ? taylor_steps(hnorm) : 0;
        S.land = land;
        S.out_idx = C->out_idx;
        S.broken = (beta > 0.0 && C->broken && m_use == C->size) ? 1 : 0;
        for (int j = 0; j <= PMAX; ++j) S.wnz[j] = j <= p ? C->wnz[j] : 0;
      }
    }
  }
  __syncwarp();

  // proposals (reading R8 of the oracle, the same arithmetic)
  if (!isfinite(omega)) {
    if (lane == 0) {
      C->status = SWE_ERR_NONFINITE;
      abort_launch(a, SWE_ERR_NONFINITE);
    }
    return;
  }
  const int cap = C->broken ? C->size : a.m_max;
  double tau_new;
  int m_new;
  if (omega == 0.0) {
    tau_new = 2.0 * tau_k;
    m_new = max(1, (3 * m_use + 3) / 4);
  } else {
    // lane 0: the step-size factor, lane 1: the Krylov-size increment
    double f = 0.0;
    if (lane == 0) f = pow(omega / a.gamma, -1.0 / fmax(1.0, m_use / 4.0));
    if (lane == 1) f = ceil(log(omega / a.gamma) / log(a.kappa));
    tau_new = tau_k * __shfl_sync(FULL, f, 0);
    tau_new = fmin(fmax(tau_new, tau_k / 5.0), 2.0 * tau_k);
    const int dm = (int)__shfl_sync(FULL, f, 1);
    m_new = m_use + dm;
    m_new = min(max(m_new, (3 * m_use + 3) / 4), (m_use * 4) / 3 + 1);
  }
  m_new = max(1, min(min(m_new, a.m_max), cap));
  const double N = 4.0 * (double)a.T.ng, nA = (double)a.nA;
  double hnorm_new = 1.0;
  if (beta > 0.0) {
    // ||tau_new Hhat||_1 = max(tau_new * max column sum of |H_m|, 1)
    hnorm_new = fmax(tau_new * sh.scal[0], 1.0);
  }
  // lane 0: C(tau_new, m), lane 1: C(tau, m_new), evaluated side by side
  const double c_lane = cost_fn(lane == 0 ? tau_new : tau_k, lane == 0 ? m_use : m_new, p, remaining, N, nA,
                                lane == 0 ? hnorm_new : hnorm);
  const double c_tau = __shfl_sync(FULL, c_lane, 0);
  const double c_m = __shfl_sync(FULL, c_lane, 1);
  if (lane != 0) return;
  const bool take_tau = (c_tau <= c_m) || (!accepted && m_new == m_use);

  // trace
  {
    DevStats* S = a.stats;
    int idx = S->n_trace;
    if (idx < a.trace_cap && a.trace != nullptr) {
      DevAttempt& r = a.trace[idx];
      r.t = t;
      r.tau = tau_k;
      r.omega = omega;
      r.m = m_use;
      r.accepted = accepted;
      r.call = a.call_index;
      r.pad = 0;
    }
    S->n_trace = idx + 1;
  }
  C->m_max_used = max(C->m_max_used, m_use);
  C->attempts += 1;
  if (replay) C->replay_pos += 1;
  C->tau_k = tau_k;
  C->land = land;
  C->accept = accepted;
  if (accepted) {
    double f = 1.0;
    for (int j = 0; j < p; ++j) {
      if (j > 0) f *= (double)j;
      C->cW[j] = tpow[j] / f;
    }
    C->ncomb = beta > 0.0 ? m_use + 1 : 0;
    C->comb_terms += C->ncomb + p;
    const double t_next = land ? t_out : t + tau_k;
    if (!(t_next > t) || C->n_sub >= a.max_substeps) {  // no progress, or too many substeps
      C->status = SWE_ERR_NOCONV;
      abort_launch(a, SWE_ERR_NOCONV);
      return;
    }
    C->t = t_next;
    C->n_sub += 1;
    if (take_tau) {
      C->tau = land ? fmax(tau_new, tau_nom) : tau_new;
    } else {
      C->tau = land ? fmax(tau_k, tau_nom) : tau_k;
      C->m = m_new;
    }
    C->m_last = m_use;
  } else {
    C->n_rej += 1;
    if (C->n_rej > a.max_reject || tau_k < 1e-14) {
      C->status = SWE_ERR_NOCONV;
      abort_launch(a, SWE_ERR_NOCONV);
      return;
    }
    if (take_tau) {
      C->tau = tau_new;
      C->m = m_use;
    } else {
      C->tau = tau_k;
      C->m = m_new;
    }
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R shared_coef(const Shared& sh, int r);
template <>
__device__ __forceinline__ double shared_coef<double>(const Shared& sh, int r) { return sh.coef[r]; }
template <>
__device__ __forceinline__ float shared_coef<float>(const Shared& sh, int r) { return sh.coeff[r]; }

// Orthogonalisation of z = A v_j against the window of raw slots lo..lo+w-1
// and pass 1 of the result at cell i (the form of orth_pass1_cell for
// windows wider than two, iom > 2): z' = z - sum_r c_r raw_{lo+r} and, by
// linearity, L z' = L z - sum_r c_r L raw_{lo+r} from the Laplacian planes
// kept for every slot.  Returns |z'|^2 of the cell.
template <typename R, bool IL>
__device__ __forceinline__ R orth_window_pass1_cell(const TablesT<R>& T, int i, const R* z, const SubBufs<R>& B,
                                                    const R* Lbuf, int lo, int w, const Shared& sh, R* rnew,
                                                    R* Lnew, const R* u, R* sq, size_t n, int p) {
  const int ng = T.ng;
  int nb[SLOTS];
  load_nbr(T, i, nb);
  R zp[4], lz[4], nrm = R(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    zp[c] = ld(z + (size_t)c * ng + i);
    lz[c] = lap_cell(T, i, nb, z + (size_t)c * ng);
  }
  for (int r = 0; r < w; ++r) {
    const R cr = shared_coef<R>(sh, r);
    const R* rr = B.raw(lo + r, n, p);
    R Lr[4];
    ld_planes<IL>(Lbuf + (size_t)(lo + r) * n, ng, i, Lr);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      zp[c] = fma(-cr, ld(rr + (size_t)c * ng + i), zp[c]);
      lz[c] = fma(-cr, Lr[c], lz[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    rnew[(size_t)c * ng + i] = zp[c];
    nrm = fma(zp[c], zp[c], nrm);
  }
  st_planes<IL>(Lnew, ng, i, lz);
  R uv[4], sv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) uv[c] = ld(u + (size_t)c * ng + i);
  sv[0] = fma(uv[0], zp[0], fma(uv[1], zp[1], fma(uv[2], zp[2], T.g * zp[3])));
#pragma unroll
  for (int c = 0; c < 3; ++c) sv[1 + c] = fma(zp[c], uv[3], uv[c] * zp[3]);
  st_planes<IL>(sq, ng, i, sv);
  return nrm;
}

// H[i][j] of the control block for any i <= j + 1.
__device__ __forceinline__ double h_entry(volatile PhiCtrl* c, int i, int j) {
  if (i == j + 1) return c->hl[j + 1];
  if (i == j) return c->hd[j];
  if (i == j - 1) return c->hu[j - 1];
  return c->hup[i * KMAX + j];
}

// Completes IOM2 column j of Algorithm 1 step 2(i) from ss = |r_{j+1}|^2, the
// squared norm of the raw vector the orthogonalisation of column j wrote:
// h_{j+1,j} = |r_{j+1}| and sig[j+1] = 1 / h_{j+1,j}, or a happy breakdown
// (invariant subspace) when h_{j+1,j} is at the rounding floor of the
// column's window coefficients.  Runs on the lane that publishes a grid
// reduction; returns false on a breakdown or a non-finite norm.
__device__ __forceinline__ bool complete_column(volatile PhiCtrl* c, GridSync* gs, int j, double ss,
                                                double bd, bool leader) {
  const double hn = sqrt(ss);
  const double ref = fabs(c->hd[j]) + (j > 0 ? fabs(c->hu[j - 1]) : 0.0);
  c->size = j + 1;
  if (leader) {
    c->n_jv += 1;
    c->n_iter += 1;
  }
  if (!isfinite(hn) || !isfinite(ref)) {
    c->status = SWE_ERR_NONFINITE;
    atomicCAS(&gs->abort, 0, SWE_ERR_NONFINITE);
    return false;
  }
  if (hn <= bd * ref) {
    c->broken = 1;
    c->hl[j + 1] = 0.0;
    c->sig[j + 1] = 0.0;
    return false;
  }
  c->hl[j + 1] = hn;
  c->sig[j + 1] = 1.0 / hn;
  return true;
}

// Algorithm 1 for one call, executed by the sh.gn blocks of a group.  Returns
// false when the launch is being aborted (every block of the group returns
// at the same barrier or at the next one).
template <typename R, bool STAGE = false>
__device__ bool phi_run(const PhiArgsT<R>& a, Shared& sh) {
  const TablesT<R>& T = a.T;
  // happy-breakdown threshold relative to the window coefficients: near the
  // rounding floor of the basis precision
  const double bd = sizeof(R) == 8 ? 1e-13 : 1e-6;
  // FP32: pass-1 planes interleaved, one 16-byte vector per cell
  constexpr bool IL = sizeof(R) == 4;
  const int ng = T.ng;
  const size_t n = (size_t)4 * ng;
  const int p = a.p;
  const int chunk = (ng + sh.gn - 1) / sh.gn;
  const Range RG{min(ng, sh.gb * chunk), min(ng, (sh.gb + 1) * chunk)};
  const CellLoop CL(RG);
  PhiCtrl* C = a.ctrl;
  // STAGE: the block's cells keep their neighbour indices in shared memory
  // for the whole launch (dynamic shared memory of SLOTS x chunk indices,
  // which the host grants; without it the indices stay in global memory).
  // Without STAGE the view stays empty and the stencils compile to their
  // global-memory loads alone.
  NbrStage ST;
  if constexpr (STAGE) {
    extern __shared__ int32_t s_nbr[];
    unsigned int dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (chunk > 0 && (size_t)dyn >= (size_t)SLOTS * chunk * sizeof(int32_t)) {
      for (int l = threadIdx.x; l < RG.c1 - RG.c0; l += blockDim.x)
#pragma unroll
        for (int k = 0; k < SLOTS; ++k) s_nbr[k * chunk + l] = __ldg(T.nbr + (size_t)k * ng + RG.c0 + l);
      __syncthreads();
      ST.s = s_nbr;
      ST.c0 = RG.c0;
      ST.stride = chunk;
    }
  }

  // ---- prologue: y = v_0, norms of the inputs -----------------------------
  if (threadIdx.x == 0) sh.t_last = globaltimer();
  if (sh.gb == 0 && threadIdx.x == 0) {
    C->status = SWE_OK;
    C->n_jv = C->n_sub = C->n_rej = C->m_last = C->m_max_used = 0;
    C->replay_pos = 0;
    C->attempts = 0;
    C->done = 0;
    C->n_iter = C->n_wjv = C->comb_terms = 0;
  }
  {
    int nz0 = 0;
    R sq[PMAX + 1];
#pragma unroll
    for (int l = 0; l <= PMAX; ++l) sq[l] = R(0);
    FOR_CELLS(i) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const size_t e = (size_t)c * ng + i;
        R yv0 = a.v[0] ? ld(a.v[0] + e) : R(0);
        (a.tapeW ? a.tapeW : a.W)[e] = yv0;
        nz0 += (yv0 != R(0)) ? 1 : 0;
        for (int l = 0; l <= p; ++l)
          if (a.v[l]) {
            R x = ld(a.v[l] + e);
            sq[l] = fma(x, x, sq[l]);
          }
      }
    }
    double v[NRED];
#pragma unroll
    for (int k = 0; k < NRED; ++k) v[k] = 0.0;
    v[0] = (double)nz0;
    for (int l = 0; l <= p; ++l) v[1 + l] = (double)sq[l];
    const int pp = p, tol_mode = a.tol_mode, m_max = a.m_max;
    const double rho0 = a.rho[0];
    const int m_init = (a.m_slot && *a.m_slot > 0) ? *a.m_slot : a.m_init;
    auto post = [pp, tol_mode, m_max, rho0, m_init](volatile PhiCtrl* c, bool, const auto& r) {
      double mx = 0.0;
#pragma unroll
      for (int l = 0; l <= PMAX; ++l)
        if (l <= pp) mx = fmax(mx, r[1 + l]);
      double scale = tol_mode == 0 ? sqrt(mx) : 1.0;
      c->scale = scale;
      c->wnz[0] = r[0] > 0.0;
      c->t = 0.0;
      c->tau = rho0;
      c->m = max(1, min(m_init, m_max));
      c->done = (scale == 0.0) || !isfinite(scale);
      if (!isfinite(scale)) c->status = SWE_ERR_NONFINITE;
    };
    if (!grid_reduce<NRED>(a, sh, v, PH_PROLOGUE, post)) return false;
  }
  if (vldi(&C->done)) {  // all inputs zero (or non-finite): zero outputs
    for (int o = 0; o < a.ns; ++o)
      FOR_CELLS(i)
        for (int c = 0; c < 4; ++c) a.y_out[o][(size_t)c * ng + i] = R(0);
    if (!grid_barrier(a, sh, PH_COMBINE)) return false;
    return vldi(&C->status) == SWE_OK;
  }

  for (int oi = 0; oi < a.ns; ++oi) {
    const double t_out = a.rho[oi];
    if (sh.gb == 0 && threadIdx.x == 0) {
      C->t_out = t_out;
      C->out_idx = oi;
    }
    while (vld(&C->t) < t_out) {
      // ---- step 1: w_j = A w_{j-1} + sum_l t^l/l! v_{j+l}  (Eq. eq3.18) ----
      const double t = vld(&C->t);
      const int ksub = vldi(&C->n_sub);
      if (a.tapeW && ksub >= a.tape_cap) {  // uniform: every block sees the same count
        if (sh.gb == 0 && threadIdx.x == 0) {
          C->status = SWE_ERR_INVALID_ARG;
          abort_launch(a, SWE_ERR_INVALID_ARG);
        }
        return false;
      }
      const SubBufs<R> B = sub_bufs(a, ksub);
      for (int j = 1; j <= p; ++j) {
        double cl[PMAX + 1];
        {
          double f = 1.0, tp = 1.0;
          for (int l = 0; l <= p - j; ++l) {
            if (l > 0) {
              f *= (double)l;
              tp *= t;
            }
            cl[l] = tp / f;
          }
        }
        const bool nz_prev = vldi(&C->wnz[j - 1]) != 0;
        R* wprev = B.Wk + (size_t)(j - 1) * n;
        R* wj = B.Wk + (size_t)j * n;
        if (nz_prev) {
          FOR_CELLS(i)
            pass1_cell<MODE_J, R, IL>(T, i, wprev, R(1), a.u_lin, a.tmp, a.tmp + (size_t)4 * ng, ST);
          if (!grid_barrier(a, sh, PH_W_PASS1)) return false;
        }
        R clr[PMAX + 1];
        for (int l = 0; l <= p - j; ++l) clr[l] = (R)cl[l];
        const R dtr = (R)a.dt;
        int nzc = 0;
        R sqs = R(0);
        FOR_CELLS(i) {
          R o[4] = {R(0), R(0), R(0), R(0)};
          if (nz_prev) pass2_cell<MODE_J, R, IL>(T, i, wprev, R(1), a.tmp, a.tmp + (size_t)4 * ng, a.aux, o, ST);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const size_t e = (size_t)c * ng + i;
            R w = dtr * o[c];
            for (int l = 0; l <= p - j; ++l)
              if (a.v[j + l]) w = fma(clr[l], ld(a.v[j + l] + e), w);
            wj[e] = w;
            nzc += (w != R(0)) ? 1 : 0;
            sqs = fma(w, w, sqs);
          }
        }
        double v[2] = {(double)nzc, (double)sqs};
        GridSync* gs = a.sync;
        auto post = [gs, j, nz_prev, p](volatile PhiCtrl* c, bool leader, const auto& r) {
          c->wnz[j] = r[0] > 0.0;
          if (nz_prev && leader) {
            c->n_jv += 1;
            c->n_wjv += 1;
          }
          if (j == p) {
            double b = sqrt(r[1]);
            c->beta = b;
            c->sig[0] = b > 0.0 ? 1.0 / b : 0.0;
            c->size = 0;
            c->broken = 0;
            if (!isfinite(b)) {
              c->status = SWE_ERR_NONFINITE;
              atomicCAS(&gs->abort, 0, SWE_ERR_NONFINITE);
            }
          }
        };
        if (!grid_reduce<2>(a, sh, v, PH_W_PASS2, post)) return false;
      }

      // ---- attempts on this substep ---------------------------------------
      while (true) {
        const double beta = vld(&C->beta);
        if (beta > 0.0) {
          int m_req;
          if (a.replay) {
            int pos = vldi(&C->replay_pos);
            m_req = pos < a.n_replay ? (int)a.replay[3 * pos + 1] : 1;
          } else {
            m_req = vldi(&C->m);
          }
          m_req = min(m_req, KMAX);
          // ---- IOM2: extend the basis to m_req columns (step 2(i)) --------
          // Per column j: pass 2 (A r_j and the two window dots) and the
          // fused orthogonalisation + pass 1 of the next vector.  Pass 2 is
          // linear, so it runs on the raw vector before its norm is known:
          // the norm's partial sums ride in the next column's reduction, and
          // the orthogonalisation ends in a plain barrier (the last column's
          // norm is reduced on its own).  Pass-1 planes of raw slot j:
          // Laplacian in Lring[j % 3], scalar/vector planes in SQ.
          R* SQ = a.tmp + (size_t)4 * ng;
          // windows wider than two (iom > 2, up to full orthogonalisation):
          // the same three phases with w window dots in one wide reduction
          while (a.iom > 2 && vldi(&C->size) < m_req && !vldi(&C->broken)) {
            const int j = vldi(&C->size);
            const int lo = max(0, j - a.iom + 1), w = j - lo + 1;
            R* rj = B.raw(j, n, p);
            R* rj1 = B.raw(j + 1, n, p);
            R* Lj = a.Lbuf + (size_t)j * n;
            R* Lj1 = a.Lbuf + (size_t)(j + 1) * n;
            const double sj = vld(&C->sig[j]);
            if (j == 0) {
              FOR_CELLS(i)
                pass1_cell<MODE_J, R, IL>(T, i, rj, R(1), a.u_lin, Lj, SQ, ST);
              if (!grid_barrier(a, sh, PH_K_PASS1)) return false;
            }
            const R zs = (R)(a.dt * sj);
            FOR_CELLS(i) {
              R o[4];
              pass2_cell<MODE_J, R, IL>(T, i, rj, R(1), Lj, SQ, a.aux, o, ST);
#pragma unroll
              for (int c = 0; c < 4; ++c) a.Zbuf[(size_t)c * ng + i] = zs * o[c];
            }
            for (int r = 0; r < w; ++r) {  // window dots <z, raw_{lo+r}>, block sums in order
              const R* rr = B.raw(lo + r, n, p);
              R acc = R(0);
              FOR_CELLS(i)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const size_t e = (size_t)c * ng + i;
                  acc = fma(a.Zbuf[e], ld(rr + e), acc);
                }
              double v1[1] = {(double)acc};
              block_sum<1>(v1, sh.red);
              if (threadIdx.x == 0) a.partw[(size_t)sh.gb * WIDE_STRIDE + r] = v1[0];
            }
            auto post_wdots = [j, lo, w](volatile PhiCtrl* c) {
              for (int r = 0; r < w; ++r) {
                const int i = lo + r;
                const double h = c->sig[i] * c->wide[r];
                if (i == j)
                  c->hd[j] = h;
                else if (i == j - 1)
                  c->hu[j - 1] = h;
                else
                  c->hup[i * KMAX + j] = h;
              }
            };
            if (!grid_reduce_wide(a, sh, w, PH_K_PASS2, post_wdots)) return false;
            for (int r = threadIdx.x; r < w; r += blockDim.x) {
              const int i = lo + r;
              sh.coef[r] = h_entry(C, i, j) * vld(&C->sig[i]);
              sh.coeff[r] = (float)sh.coef[r];
            }
            __syncthreads();
            R nrm = R(0);
            FOR_CELLS(i)
              nrm += orth_window_pass1_cell<R, IL>(T, i, a.Zbuf, B, a.Lbuf, lo, w, sh, rj1, Lj1, a.u_lin, SQ, n, p);
            double wn[1] = {(double)nrm};
            GridSync* gs = a.sync;
            auto post_wnorm = [gs, j, lo, w, bd](volatile PhiCtrl* c, bool leader, const auto& r) {
              double hn = sqrt(r[0]);
              double ref = 0.0;
              for (int r = 0; r < w; ++r) ref += fabs(h_entry(c, lo + r, j));
              c->size = j + 1;
              if (leader) {
                c->n_jv += 1;
                c->n_iter += 1;
              }
              if (!isfinite(hn) || !isfinite(ref)) {
                c->status = SWE_ERR_NONFINITE;
                atomicCAS(&gs->abort, 0, SWE_ERR_NONFINITE);
                return;
              }
              if (hn <= bd * ref) {  // happy breakdown: invariant subspace
                c->broken = 1;
                c->hl[j + 1] = 0.0;
                c->sig[j + 1] = 0.0;
              } else {
                c->hl[j + 1] = hn;
                c->sig[j + 1] = 1.0 / hn;
              }
            };
            if (!grid_reduce<1>(a, sh, wn, PH_ORTH, post_wnorm)) return false;
          }
          if (vldi(&C->size) < m_req && !vldi(&C->broken)) {
            int j = vldi(&C->size);
            R nrm = R(0);      // this thread's share of |r_j|^2 while column j-1 is open
            bool pend = false;  // column j-1 open: its norm joins column j's reduction
            GridSync* gs = a.sync;
            const double dt = a.dt;
            while (true) {
              R* rj = B.raw(j, n, p);
              R* rj1 = B.raw(j + 1, n, p);
              R* rjm = j > 0 ? B.raw(j - 1, n, p) : nullptr;
              R* Lj = a.Lring + (size_t)(j % 3) * n;
              R* Ljm = a.Lring + (size_t)((j + 2) % 3) * n;
              R* Lj1 = a.Lring + (size_t)((j + 1) % 3) * n;
              if (j == 0) {
                FOR_CELLS(i)
                  pass1_cell<MODE_J, R, IL>(T, i, rj, R(1), a.u_lin, Lj, SQ, ST);
                if (!grid_barrier(a, sh, PH_K_PASS1)) return false;
              }
              // pass 2: A r_j of the raw vector (its scale may not be known yet)
              R d0 = R(0), d1 = R(0);
              FOR_CELLS(i) {
                R o[4];
                pass2_cell<MODE_J, R, IL>(T, i, rj, R(1), Lj, SQ, a.aux, o, ST);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const size_t e = (size_t)c * ng + i;
                  a.Zbuf[e] = o[c];
                  if (rjm) d0 = fma(o[c], rjm[e], d0);
                  d1 = fma(o[c], rj[e], d1);
                }
              }
              // one reduction: |r_j|^2 (closing column j-1), <A r_j, r_{j-1}>, <A r_j, r_j>
              double v[3] = {(double)nrm, (double)d0, (double)d1};
              auto post_col = [gs, j, pend, bd, dt](volatile PhiCtrl* c, bool leader, const auto& r) {
                if (pend && !complete_column(c, gs, j - 1, r[0], bd, leader)) return;
                const double sj = c->sig[j];
                const double zs = dt * sj;  // z = zs A r_j = dt A v_j
                if (j > 0) c->hu[j - 1] = c->sig[j - 1] * (zs * r[1]);
                c->hd[j] = sj * (zs * r[2]);
              };
              if (!grid_reduce<3>(a, sh, v, PH_K_PASS2, post_col)) return false;
              if (vldi(&C->broken)) break;  // column j-1 ended the basis; A r_j unused
              // z' = z - h_{j-1,j} v_{j-1} - h_{j,j} v_j with its pass-1 planes
              const double sj = vld(&C->sig[j]);
              const double sjm = j > 0 ? vld(&C->sig[j - 1]) : 0.0;
              const R zs = (R)(dt * sj);
              const R am = j > 0 ? (R)(vld(&C->hu[j - 1]) * sjm) : R(0);
              const R aj = (R)(vld(&C->hd[j]) * sj);
              nrm = R(0);
              FOR_CELLS(i)
                nrm += orth_pass1_cell<R, IL>(T, i, a.Zbuf, zs, rj, rjm, aj, am, Lj, Ljm, rj1, Lj1, a.u_lin, SQ, ST);
              if (j + 1 < m_req) {  // pass 2 of r_{j+1} needs its planes on every cell
                if (!grid_barrier(a, sh, PH_ORTH)) return false;
                pend = true;
                ++j;
                continue;
              }
              double w[1] = {(double)nrm};
              auto post_last = [gs, j, bd](volatile PhiCtrl* c, bool leader, const auto& r) {
                complete_column(c, gs, j, r[0], bd, leader);
              };
              if (!grid_reduce<1>(a, sh, w, PH_ORTH, post_last)) return false;
              break;
            }
          }
        }
        // ---- exponential, error estimate, controller (steps 2(ii)-6) -------
        if (sh.gb == 0) decide(a, sh);
        if (!grid_barrier(a, sh, PH_DECIDE)) return false;
        if (!vldi(&C->accept)) continue;

        // ---- y_{k+1} = tau^p phi_p(tau A) w_p + sum_{j<p} tau^j/j! w_j (eq3.17)
        const int ncomb = vldi(&C->ncomb);
        for (int r = threadIdx.x; r < ncomb; r += blockDim.x) {
          sh.coef[r] = vld(&C->cV[r]);
          sh.coeff[r] = (float)sh.coef[r];
        }
        for (int r = threadIdx.x; r < p; r += blockDim.x) {
          sh.coef[KMAX + 2 + r] = vld(&C->cW[r]);
          sh.coeff[KMAX + 2 + r] = (float)sh.coef[KMAX + 2 + r];
        }
        __syncthreads();
        const bool land = vldi(&C->land) != 0;
        R* yo = land ? a.y_out[oi] : nullptr;
        int nzy = 0;
        // Per element the sum runs over w_0..w_{p-1}, then raw slots 0..ncomb-1,
        // one FMA each in that order; a thread loads kQ slots x four
        // components of its cell before it uses them, so that enough loads are
        // in flight to cover the memory latency (kQ = 4 within the FP32
        // kernel's 64 registers).
        constexpr int kQ = sizeof(R) == 8 ? 8 : 4;
        FOR_CELLS(i) {
          R y[4] = {R(0), R(0), R(0), R(0)};
          for (int j = 0; j < p; ++j) {
            const R cj = shared_coef<R>(sh, KMAX + 2 + j);
            const R* src = B.Wk + (size_t)j * n + i;
            R wv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) wv[c] = src[(size_t)c * ng];
#pragma unroll
            for (int c = 0; c < 4; ++c) y[c] = fma(cj, wv[c], y[c]);
          }
          int r = 0;
          for (; r + kQ <= ncomb; r += kQ) {
            R xv[kQ][4];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
              const R* src = B.raw(r + q, n, p) + i;
#pragma unroll
              for (int c = 0; c < 4; ++c) xv[q][c] = src[(size_t)c * ng];
            }
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
              const R cq = shared_coef<R>(sh, r + q);
#pragma unroll
              for (int c = 0; c < 4; ++c) y[c] = fma(cq, xv[q][c], y[c]);
            }
          }
          for (; r < ncomb; ++r) {
            const R cr = shared_coef<R>(sh, r);
            const R* src = B.raw(r, n, p) + i;
#pragma unroll
            for (int c = 0; c < 4; ++c) y[c] = fma(cr, src[(size_t)c * ng], y[c]);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const size_t e = (size_t)c * ng + i;
            B.Wnext[e] = y[c];
            if (yo) yo[e] = y[c];
            nzy += (y[c] != R(0)) ? 1 : 0;
          }
        }
        double v[1] = {(double)nzy};
        auto post_y = [](volatile PhiCtrl* c, bool, const auto& r) { c->wnz[0] = r[0] > 0.0; };
        if (!grid_reduce<1>(a, sh, v, PH_COMBINE, post_y)) return false;
        break;
      }
    }
  }

  return true;
}

// Statistics of one call, written by block 0 of the group once the call has
// ended (normally or by abort).
template <typename R>
__device__ void phi_finish(const PhiArgsT<R>& a, Shared& sh) {
  const int ng = a.T.ng;
  PhiCtrl* C = a.ctrl;
  if (sh.gb == 0 && threadIdx.x == 0) {
    DevStats* S = a.stats;
    int ab = ld_volatile_int(&a.sync->abort);
    int st = C->status != SWE_OK ? C->status : ab;
    S->n_jv += C->n_jv;
    S->n_iter += C->n_iter;
    S->n_wjv += C->n_wjv;
    S->comb_terms += C->comb_terms;
    S->n_sub += C->n_sub;
    S->n_rej += C->n_rej;
    S->m_last = C->m_last;
    S->m_max_used = max(S->m_max_used, C->m_max_used);
    if (S->status == SWE_OK) S->status = st;
    if (a.m_slot && st == SWE_OK && C->m_last > 0) *a.m_slot = C->m_last;
    if (a.prof) {
      // per cell: IOM2 iteration 346 flop / 136 B, w_j product 310 / 104,
      // combination term 8 / 32 (bytes of FP64 vectors; FP32 vectors move half)
      const double cells = (double)ng, esz = (double)sizeof(R) / 8.0;
      a.prof->iters += C->n_iter;
      a.prof->wjv += C->n_wjv;
      a.prof->comb_terms += C->comb_terms;
      a.prof->launches += 1;
      a.prof->flop += cells * (kFlopIter * C->n_iter + kFlopWjv * C->n_wjv + kFlopComb * C->comb_terms);
      a.prof->bytes += cells * esz * (136.0 * C->n_iter + 104.0 * C->n_wjv + 32.0 * C->comb_terms);
      // tables: a pass 1 and a pass 2 per IOM2 iteration and per w_j product
      a.prof->table_bytes += cells * (62.0 * sizeof(R) + 48.0) * (double)(C->n_iter + C->n_wjv);
    }
  }
}

// ---------------------------------------------------------------------------
// Ensemble launch: every member's group of blocks advances its exprb42
// trajectory (stage passes, both phipm_simul_iom2 calls and the update) for
// nsteps steps.  Members never wait on one another; each group has its own
// barrier, control block and reduction buffer, so a member that stops (error)
// does not hold the others.  A group may hold several members, run one after
// the other on the same blocks (small members stacked so that they share
// blocks instead of idling on one each).
// ---------------------------------------------------------------------------
__device__ bool ens_step(const EnsMember& M, Shared& sh) {
  const Tables& T = M.c1.T;
  const int ng = T.ng;
  const int chunk = (ng + sh.gn - 1) / sh.gn;
  const Range RG{min(ng, sh.gb * chunk), min(ng, (sh.gb + 1) * chunk)};
  const CellLoop CL(RG);
  double* S1 = M.tmpS;
  double* S2 = M.tmpS + (size_t)4 * ng;
  // eta, n x u of u_n and pass 1 of F(u_n)
  FOR_CELLS(i) {
    aux_cell(T, i, (const double*)M.u, M.aux);
    pass1_cell<MODE_F>(T, i, (const double*)M.u, 1.0, (const double*)nullptr, S1, S2);
  }
  if (!grid_barrier(M.c1, sh, PH_PROLOGUE)) return false;
  FOR_CELLS(i) {
    double o[4];
    pass2_cell<MODE_F>(T, i, (const double*)M.u, 1.0, S1, S2, (const double*)nullptr, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) M.vF[(size_t)c * ng + i] = M.dt * o[c];
  }
  if (!grid_barrier(M.c1, sh, PH_PROLOGUE)) return false;
  // U_n2 - u_n = (3/4) dt phi_1((3/4) dt J) F(u_n)
  bool ok = phi_run<double>(M.c1, sh);
  phi_finish<double>(M.c1, sh);
  if (!ok) return false;
  // D_n2 = N(U_n2) - N(u_n) = Q(U_n2 - u_n); v_3 = (32/9) dt D_n2
  FOR_CELLS(i) pass1_cell<MODE_Q>(T, i, (const double*)M.y1, 1.0, (const double*)nullptr, S1, S2);
  if (!grid_barrier(M.c1, sh, PH_PROLOGUE)) return false;
  const double c3 = (32.0 / 9.0) * M.dt;
  FOR_CELLS(i) {
    double o[4];
    pass2_cell<MODE_Q>(T, i, (const double*)M.y1, 1.0, S1, S2, (const double*)nullptr, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) M.v3[(size_t)c * ng + i] = c3 * o[c];
  }
  if (!grid_barrier(M.c1, sh, PH_PROLOGUE)) return false;
  // w = phi_1(A) v + phi_3(A) (32/9) dt D_n2; u_{n+1} = u_n + w
  ok = phi_run<double>(M.c2, sh);
  phi_finish<double>(M.c2, sh);
  if (!ok) return false;
  FOR_CELLS(i) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const size_t e = (size_t)c * ng + i;
      M.u[e] = M.u[e] + M.w[e];
    }
  }
  return grid_barrier(M.c1, sh, PH_PROLOGUE);
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) ens_kernel(EnsMember* __restrict__ mem, const int* __restrict__ blk2mem) {
  __shared__ Shared sh;
  for (int m = blk2mem[blockIdx.x]; m >= 0; m = mem[m].next) {
    EnsMember& M = mem[m];
    if (threadIdx.x == 0) {
      sh.gb = blockIdx.x - M.b0;
      sh.gn = M.nb;
      if (sh.gb == 0) M.t0 = globaltimer();
    }
    __syncthreads();
    for (int s = 0; s < M.nsteps; ++s)
      if (!ens_step(M, sh)) break;
    if (threadIdx.x == 0 && sh.gb == 0) M.t1 = globaltimer();
    __syncthreads();
  }
}

// Launch shapes of the ensemble kernel: block size x resident blocks per SM
// (the same 384 threads per SM, 168 registers each); the block size sets the
// granularity of the split between members.
struct EnsVariant {
  const void* fn;
  int threads;
};
static const EnsVariant kEnsVariants[ENS_SHAPES] = {
    {(const void*)ens_kernel<96, 4>, 96},
    {(const void*)ens_kernel<128, 3>, 128},
    {(const void*)ens_kernel<192, 2>, 192},
    {(const void*)ens_kernel<384, 1>, 384},
};

int ens_max_blocks(int shape, int* nblocks, int* threads, int* per_sm) {
  if (shape < 0 || shape >= ENS_SHAPES) return -1;
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const EnsVariant& v = kEnsVariants[shape];
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, v.fn, v.threads, 0) != cudaSuccess || per < 1)
    return -1;
  *nblocks = per * nsm;
  *threads = v.threads;
  if (per_sm) *per_sm = per;
  return 0;
}

int launch_ens_kernel(int shape, EnsMember* mem, const int* blk2mem, int nblocks, cudaStream_t stream) {
  if (shape < 0 || shape >= ENS_SHAPES) return (int)cudaErrorInvalidValue;
  const EnsVariant& v = kEnsVariants[shape];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(v.threads);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&mem, (void*)&blk2mem};
  cudaError_t e = cudaLaunchKernelExC(&cfg, v.fn, args);
  return e == cudaSuccess ? 0 : (int)e;
}

// Instantiations (block size, minimum resident blocks per SM for the register
// budget).  The body adapts to blockDim.x; the taylor exponential needs at
// least m_max + p + 1 = 69 threads.
template <typename R, int NT, int MINB, bool STAGE = false>
__global__ void __launch_bounds__(NT, MINB) phi_kernel(const __grid_constant__ PhiArgsT<R> a) {
  static_assert(NT % 32 == 0 && NT <= PHI_MAX_THREADS, "block size beyond the shared reduction scratch");
  __shared__ Shared sh;
  if (threadIdx.x == 0) {
    sh.gb = blockIdx.x;
    sh.gn = gridDim.x;
  }
  __syncthreads();
  phi_run<R, STAGE>(a, sh);
  phi_finish<R>(a, sh);
}

struct PhiVariant {
  const void* fn;
  int threads;
};
static const PhiVariant kVariantsF64[] = {
    {(const void*)phi_kernel<double, 384, 1>, 384},
    {(const void*)phi_kernel<double, 256, 2>, 256},
    {(const void*)phi_kernel<double, 192, 2>, 192},
    {(const void*)phi_kernel<double, 128, 3>, 128},
    {(const void*)phi_kernel<double, 96, 4>, 96},
};
// One FP32 shape: two 512-thread blocks per SM hold the most threads at the
// 64 registers the stencils fit in, which is how single-precision shapes are
// ranked (below); smaller shapes never rank first and are not built.
static const PhiVariant kVariantsF32[] = {
    {(const void*)phi_kernel<float, 512, 2>, 512},
};

// Instantiations whose blocks keep their neighbour indices in shared memory,
// beside the plain ones they replace when the indices fit.  Only the FP32
// stencils, bound by the latency of the index -> gather chain, have one; the
// FP64 stencils are bound by the FP64 unit and run no faster staged.
struct PhiStaged {
  const void* plain;
  const void* staged;
};
static const PhiStaged kStaged[] = {
    {(const void*)phi_kernel<float, 512, 2>, (const void*)phi_kernel<float, 512, 2, true>},
};

// Picks the instantiation and block count for a grid of ng cells.  The FP64
// unit charges a whole warp slot per warp instruction however many lanes are
// active, so the cost of a stencil phase on the busiest SM is proportional to
// (resident blocks) x (rounds of blockDim cells per block) x (warps per
// block); the variant with the fewest such warp-rounds wins (ties: the
// earlier, larger block, i.e. fewer barrier participants).  The FP32 stencils are bound by
// memory latency instead (the FP32 pipe is 64x the FP64 one), so the single
// precision variants are ranked by resident threads per SM (more loads in
// flight), then by fewer blocks (cheaper barriers).  Small grids use fewer
// blocks.
int phi_select(int ng, int single, PhiLaunch* out) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  long long best = 0;
  bool found = false;
  const PhiVariant* vs = single ? kVariantsF32 : kVariantsF64;
  const int nv = single ? (int)(sizeof(kVariantsF32) / sizeof(kVariantsF32[0]))
                        : (int)(sizeof(kVariantsF64) / sizeof(kVariantsF64[0]));
  for (int q = 0; q < nv; ++q) {
    const PhiVariant& v = vs[q];
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, v.fn, v.threads, 0) != cudaSuccess || per < 1)
      continue;
    long long nb = (long long)per * nsm;
    long long need = (ng + v.threads - 1) / v.threads;
    if (need < nb) nb = need;
    if (nb < 1) nb = 1;
    long long cells = (ng + nb - 1) / nb;
    long long rounds = (cells + v.threads - 1) / v.threads;
    long long per_sm = (nb + nsm - 1) / nsm;
    long long cost = single ? -((long long)per * v.threads * 4096 - nb) : per_sm * rounds * (v.threads / 32);
    if (!found || cost < best) {
      found = true;
      best = cost;
      out->fn = v.fn;
      out->threads = v.threads;
      out->nblocks = (int)nb;
    }
  }
  if (!found) return -1;
  // Each block's neighbour indices go to shared memory when the variant has a
  // staged instantiation and they fit without lowering the occupancy the
  // variant was ranked with.  The function's dynamic shared memory limit is
  // raised to the device maximum (grids of other sizes share the function);
  // the launch asks for what it needs.
  out->smem = 0;
  const void* staged = nullptr;
  for (const PhiStaged& st : kStaged)
    if (st.plain == out->fn) staged = st.staged;
  if (!staged) return 0;
  const long long chunk = (ng + out->nblocks - 1) / out->nblocks;
  const long long need = (long long)SLOTS * chunk * (long long)sizeof(int32_t);
  int optin = 0;
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
      cudaFuncGetAttributes(&fa, staged) == cudaSuccess && need + (long long)fa.sharedSizeBytes <= optin &&
      cudaFuncSetAttribute(staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes) == cudaSuccess) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, staged, out->threads, (size_t)need) == cudaSuccess &&
        (long long)per * nsm >= out->nblocks) {
      out->fn = staged;
      out->smem = (int)need;
    }
  }
  (void)cudaGetLastError();  // a refused attribute only leaves the indices in global memory
  return 0;
}

// Cooperative launch (all blocks co-resident: the grid barriers need it).
template <class A>
int launch_phi_kernel(const PhiLaunch& L, const A& a, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.nblocks);
  cfg.blockDim = dim3(L.threads);
  cfg.dynamicSmemBytes = (size_t)L.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&a};
  cudaError_t e = cudaLaunchKernelExC(&cfg, L.fn, args);
  return e == cudaSuccess ? 0 : (int)e;
}
template int launch_phi_kernel<PhiArgs>(const PhiLaunch&, const PhiArgs&, cudaStream_t);
template int launch_phi_kernel<PhiArgsF>(const PhiLaunch&, const PhiArgsF&, cudaStream_t);

}  // namespace swe
