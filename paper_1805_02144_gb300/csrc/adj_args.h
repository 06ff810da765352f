// Arguments and control block of the adjoint launch (adj_kernel.cu).
#pragma once
#include <stdint.h>

#include "phi_args.h"
#include "swe_dev.cuh"

namespace swe {

constexpr int ADJ_KW = KMAX + 4;  // stride of the wide reduction's partial sums

// Written by one block between grid barriers, read by all (volatile reads).
struct AdjCtrl {
  double red[NRED];          // last narrow reduction
  double wide[ADJ_KW];       // last wide reduction: <r_r, Y> (r <= m), two basis dots
  double alpha[KMAX + 2];    // Y-coefficient of Vbar_r (update of Eq. eq3.17)
  double hdb[KMAX + 1];      // adjoint of H[j][j]
  double hub[KMAX + 1];      // adjoint of H[j][j+1]
  double hlb[KMAX + 2];      // adjoint of H[j][j-1] (hlb[m]: of h_{m+1,m})
  double betabar;
  double col[4];             // etabar, abar, bbar of the next column; <Vbar_0, v_0>
  int status, pad;
};

// One adjoint launch: the reverse of one phipm_simul_iom2 call recorded on a
// tape (see PhiArgsT).  Accumulates into vbar[l] (nullable) and ubar.
struct AdjArgs {
  Tables T;                  // FP64 tables including the transposed ones
  const double* u_lin;       // linearisation state u_n
  const double* aux;         // eta (with f) and n x u of u_lin
  double dt;
  int p, nsub, ns;
  const double* ybar[NSMAX]; // adjoints of the outputs y(rho_i); nullptr = 0
  double* vbar[PMAX + 1];    // += adjoints of v_0..v_p (nullable)
  double* ubar;              // += dt sum Q'(x)^T xbar over every product A x
  // tape of the forward call
  const double* tapeW;
  const double* tapeV;
  const long long* tape_offV;
  const long long* tape_mmax;  // largest m each substep's basis region holds
  const TapeSub* tape_sub;
  int* status_out;           // nullable: the launch's status is stored here at exit
  // workspace
  double* Y;                 // n: adjoint of the current substep's output
  double* Wb;                // (PMAX + 1) n: adjoints of w_j
  double* X;                 // 2 n: completed basis adjoints (ring)
  double* P;                 // 2 n: partial basis adjoints (ring)
  double* PL;                // 10 ng: transposed pass-1 planes
  double* Zb;                // n: the vector being transposed
  double* part;              // NRED x nblocks (value-major)
  double* partw;             // nblocks x ADJ_KW
  double* xs;                // (xs_steps + TAYLOR + 1) x (KMAX + PMAX + 2)
  int xs_steps;
  AdjCtrl* ctrl;
  GridSync* sync;
  DevProfile* prof;          // nullable (phase timing is not collected here)
};

}  // namespace swe
