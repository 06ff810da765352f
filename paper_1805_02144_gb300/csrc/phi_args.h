// Arguments and device control block of the persistent phipm_simul_iom2 launch.
#pragma once
#include <stdint.h>

#include "swe_dev.cuh"

namespace swe {

constexpr int KMAX = 64;   // largest Krylov size
constexpr int PMAX = 4;    // largest phi index p
constexpr int NSMAX = 8;   // largest number of outputs rho_i
constexpr int NRED = 8;    // values per grid reduction

// Statistics accumulated on the device over one phi_action or one exprb_step.
struct DevStats {
  int n_jv, n_sub, n_rej, m_last, m_max_used, status, n_trace, pad;
  long long n_iter, n_wjv, comb_terms;  // IOM2 columns, w_j products, combination terms
};

// Operation counters accumulated while profiling is on.
struct DevProfile {
  long long iters, wjv, comb_terms, launches;
  long long phase_ns[10];  // block 0's time per phase class (see phi_kernel.cu)
  double flop, bytes;      // algorithmic operation count and vector bytes of the launches
  double table_bytes;      // operator-table bytes the launches read
};

// One trace record, the same layout as the public phi_attempt.
struct DevAttempt {
  double t, tau, omega;
  int m, accepted, call, pad;
};

// Control block written by one thread between grid barriers and read by all.
struct PhiCtrl {
  double red[NRED];
  double hd[KMAX + 1];      // H[j][j]
  double hu[KMAX + 1];      // H[j][j+1]
  double hl[KMAX + 2];      // H[j][j-1]; hl[m] is h_{m+1,m} of an m-column basis
  double sig[KMAX + 2];     // basis vector j = sig[j] * raw slot j
  double cV[KMAX + 2];      // combination coefficients of raw slots 0..m
  double cW[PMAX + 1];      // combination coefficients of w_0..w_{p-1}
  double beta, scale;
  double t, tau, tau_k, t_out;
  int size, broken, m, ncomb;
  int land, accept, out_idx, done;
  int wnz[PMAX + 1];
  int n_jv, n_sub, n_rej, m_last, m_max_used, status, replay_pos, attempts;
  int n_iter, n_wjv, comb_terms, pad;
  // wider orthogonalisation windows (iom > 2): the dots of the last wide
  // reduction and H[i][j] for i <= j - 2 (row-major, KMAX columns)
  double wide[KMAX + 4];
  double hup[KMAX * KMAX];
};

constexpr int WIDE_STRIDE = KMAX + 4;  // per-block stride of wide partial sums

// Scalars of one accepted substep kept for the adjoint (tape mode).
struct TapeSub {
  double t, tau, beta, hnext;
  int m, s, land, out_idx;  // s: scaling steps of the exponential
  int broken, pad0;
  int wnz[PMAX + 1];        // w_j != 0 (zero skip of Eq. eq3.18)
  int pad1;
  double sig[KMAX + 2];     // basis vector j = sig[j] * raw slot j
  double hd[KMAX + 1], hu[KMAX + 1], hl[KMAX + 2];
};

// The persistent-kernel instantiation chosen for a grid.
struct PhiLaunch {
  const void* fn = nullptr;
  int threads = 0;
  int nblocks = 0;
  int smem = 0;  // dynamic shared memory: the blocks' neighbour indices (0: read from global)
};

// Arguments of one persistent launch.  R is the precision of tables, vectors
// and stencil arithmetic (double: FP64 path; float: mixed path, whose
// reductions, control block, exponential and controller stay in double).
template <typename R>
struct PhiArgsT {
  TablesT<R> T;
  const R* u_lin;           // [4][ng] linearisation state (read-only)
  const R* aux;             // [4][ng] eta and n x u of u_lin
  double dt;
  int p, ns;
  double rho[NSMAX];
  const R* v[PMAX + 1];     // device, nullptr = zero
  R* y_out[NSMAX];
  // workspace
  R* Vbuf;                  // (KMAX + 1) raw basis slots of n values (slot 0 unused)
  R* W;                     // (PMAX + 1) x n: W[0] = y_k, W[j] = w_j
  R* tmp;                   // 8 x ng pass-1 planes (Laplacian 4, scalar/vector 4)
  R* Lring;                 // 3 x n: Laplacian planes of the last three raw slots
  R* Zbuf;                  // n: A v_j before orthogonalisation
  R* Lbuf;                  // iom > 2: (KMAX + 1) x n Laplacian planes of every raw slot
  double* partw;            // iom > 2: nblocks x WIDE_STRIDE partial dots
  double* part;             // NRED x nblocks partial sums (value-major)
  PhiCtrl* ctrl;
  GridSync* sync;
  DevStats* stats;          // accumulated (not reset by the kernel)
  DevProfile* prof;         // nullable: operation counters
  DevAttempt* trace;        // capacity trace_cap, appended at stats->n_trace
  int trace_cap;
  int call_index;
  int* m_slot;              // nullable: initial m (if > 0), receives m_last
  const double* replay;     // nullable device array, 3 doubles per attempt
  int n_replay;
  // tape (adjoint recording, nullptr = off).  Accepted substep k keeps w_j in
  // tapeW + k (p+1) n + j n and raw basis slot j >= 1 in tapeV + tape_offV[k]
  // + j n; y_{k+1} is written to slot 0 of region k + 1.
  R* tapeW;
  R* tapeV;
  const long long* tape_offV;
  TapeSub* tape_sub;
  int tape_cap;             // accepted substeps the tape holds
  // options
  double tol, delta, gamma, kappa;
  int tol_mode, m_init, m_max, max_reject, max_substeps;
  int iom;                  // orthogonalisation window (2: IOM2; up to KMAX: full)
  int64_t nA;
};
using PhiArgs = PhiArgsT<double>;
using PhiArgsF = PhiArgsT<float>;

constexpr int ENS_SHAPES = 4;  // launch shapes of the ensemble kernel (96x4, 128x3, 192x2, 384x1)

// Algorithmic FP64 operations per cell (FMA = 2), counted from the stencils:
// one IOM2 column (pass 1 + pass 2 of J x, two window dots, the
// orthogonalisation and its norm), one w_j product (J x and the combination
// of Eq. eq3.18), one term of the substep combination (Eq. eq3.17).
constexpr double kFlopIter = 346.0, kFlopWjv = 310.0, kFlopComb = 8.0;

// One member of an ensemble launch: an exprb42 trajectory (Eq. eq3.11 with
// the two phipm_simul_iom2 calls of Sec. 4.4) advanced nsteps steps by the
// group of blocks [b0, b0 + nb).
struct EnsMember {
  PhiArgs c1;               // p = 1, rho = {3/4}: Y(3/4) = U_n2 - u_n  -> y1
  PhiArgs c2;               // p = 3, rho = {1}, v_1 = dt F, v_3 = (32/9) dt D_n2 -> w
  double* u;                // state (library-owned), n values
  double* vF;               // dt F(u_n)
  double* v3;               // (32/9) dt D_n2
  double* y1;               // = c1.y_out[0]
  double* w;                // = c2.y_out[0]
  double* tmpS;             // 8 planes for the F and Q passes
  double* aux;              // = c1.aux (written here)
  double dt;
  int nsteps;
  int b0, nb;
  int next;                   // the member that runs next on the same blocks, or -1
  int pad;
  unsigned long long t0, t1;  // globaltimer at the member's start and end (block 0)
};

}  // namespace swe
