// C ABI of the library (include/swe_exprb.h): grid handles, the F / J x
// stencil kernels, phi_action (one persistent launch of phipm_simul_iom2) and
// the exprb_step drivers of Sec. 4.4.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/swe_exprb.h"
#include "adj_args.h"
#include "grid_build.h"
#include "phi_args.h"
#include "swe_dev.cuh"

namespace swe {
int adj_max_blocks(int* nblocks, int* threads);
int launch_adj_kernel(const AdjArgs& a, int nblocks, cudaStream_t st);
template <class A>
int launch_phi_kernel(const PhiLaunch& L, const A& a, cudaStream_t stream);
int phi_select(int ng, int single, PhiLaunch* out);
int ens_max_blocks(int shape, int* nblocks, int* threads, int* per_sm);
int launch_ens_kernel(int shape, EnsMember* mem, const int* blk2mem, int nblocks, cudaStream_t stream);
}  // namespace swe

using namespace swe;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(SWE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int TRACE_CAP = 4096;
constexpr int STAGE_VECS = 12;

}  // namespace

// ---------------------------------------------------------------------------
// grid handle
// ---------------------------------------------------------------------------
struct swe_grid {
  HostGrid host;
  Tables T;
  int device = 0;
  void* dtab = nullptr;      // one allocation for all tables
  // workspace (lazily allocated)
  void* dws = nullptr;
  size_t ws_bytes = 0;
  double* Vbuf = nullptr;
  double* W = nullptr;
  double* tmp = nullptr;
  double* tmp2 = nullptr;
  double* Lring = nullptr;
  double* Zbuf = nullptr;
  double* aux = nullptr;
  double* part = nullptr;
  double* stage = nullptr;   // STAGE_VECS vectors of n
  PhiCtrl* ctrl = nullptr;
  GridSync* sync = nullptr;
  DevStats* stats = nullptr;
  DevAttempt* trace = nullptr;
  double* replay = nullptr;
  int replay_cap = 0;
  PhiLaunch launch;          // persistent-kernel instantiation for this grid (FP64)
  // mixed precision (created on first use)
  TablesF TF;
  void* dtabF = nullptr;
  void* dwsF = nullptr;
  PhiLaunch launchF;
  float *VbufF = nullptr, *WF = nullptr, *tmpF = nullptr, *LringF = nullptr, *ZbufF = nullptr,
        *auxF = nullptr, *ulinF = nullptr, *vinF = nullptr, *youtF = nullptr;
  size_t tab_bytes = 0;      // size of the table allocation
  // profiling (swe_profile_enable)
  bool prof_on = false;
  DevProfile* dprof = nullptr;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> phi_ev, call_ev;
  int64_t kernel_launches = 0;
  // adjoint (created on first use)
  void* dadj = nullptr;
  int adj_nblocks = 0;
  double *aY = nullptr, *aWb = nullptr, *aX = nullptr, *aP = nullptr, *aPL = nullptr, *aZb = nullptr,
         *apart = nullptr, *apartw = nullptr, *axs = nullptr, *avec = nullptr;
  AdjCtrl* actrl = nullptr;
  void* dtape = nullptr;     // tapes of the recorded forward calls (grown on demand)
  size_t tape_bytes = 0;
  long long* hstage = nullptr;  // pinned staging of the tape layout (offsets, sizes)
  size_t hstage_cap = 0;
  cudaEvent_t stage_ev = nullptr;
  int* adj_status = nullptr;    // device: first error of the adjoint launches of a step
  double* dhs = nullptr;        // surface height h_s (device), when set
  // windows wider than two (iom > 2): Laplacian planes of every basis slot
  // and wide partial sums, per precision, created on first use
  void* dwide = nullptr;
  void* dwideF = nullptr;
};

struct swe_ensemble {
  int nmem = 0;
  int shape = 0;              // launch shape (index of the ensemble kernel variant)
  int nblocks = 0;            // blocks of the launch (all co-resident)
  int nb_alloc = 0;           // the most blocks any shape launches (sizes dblk, part)
  std::vector<swe_grid*> grids;
  std::vector<EnsMember> hmem;
  std::vector<std::vector<int>> groups;  // members run back to back on one group of blocks
  std::vector<int> gnb;       // blocks per group
  std::vector<int> nb;        // blocks per member (its group's)
  std::vector<double> weight; // work model per member (cells x 2^level x simulated time)
  EnsMember* dmem = nullptr;
  int* dblk = nullptr;        // block -> member
  GridSync* dsync = nullptr;  // nmem
  DevStats* dstats = nullptr; // nmem
  void* dws = nullptr;        // member workspaces
  double* backup = nullptr;   // states saved while tuning
  std::vector<size_t> state_off;  // offset of member m's state in backup (doubles)
  int* dslots = nullptr;      // 2 per member: Krylov size carried between steps and runs
  int* dslots_backup = nullptr;
};

struct swe_scheme_state {
  const swe_grid* grid = nullptr;
  double* u_prev = nullptr;  // epi3 history (device)
  int* m_slots = nullptr;    // device ints, one per call slot
  int have_prev = 0;
};

namespace {

// ---------------------------------------------------------------------------
// standalone kernels
// ---------------------------------------------------------------------------
constexpr int TPB = 256;

template <typename R>
__global__ void k_aux(TablesT<R> T, const R* __restrict__ u, R* aux) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.ng; i += gridDim.x * blockDim.x)
    aux_cell(T, i, u, aux);
}

template <int MODE>
__global__ void k_pass1(Tables T, const double* x, double sx, const double* u, double* tmp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.ng; i += gridDim.x * blockDim.x)
    pass1_cell<MODE>(T, i, x, sx, u, tmp, tmp + (size_t)4 * T.ng);
}

// out = alpha * stencil(x)  (+ beta_ * add, when add != nullptr)
template <int MODE>
__global__ void k_pass2(Tables T, const double* x, double sx, const double* tmp, const double* aux,
                        double alpha, double* out) {
  const int ng = T.ng;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
    double o[4];
    pass2_cell<MODE>(T, i, x, sx, tmp, tmp + (size_t)4 * ng, aux, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) out[(size_t)c * ng + i] = alpha * o[c];
  }
}

template <int MODE>
__global__ void k_pass1T(Tables T, const double* lam, const double* aux, double* t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.ng; i += gridDim.x * blockDim.x)
    pass1T_cell<MODE>(T, i, lam, aux, t);
}

// out = alpha * stencil (accumulate = 0) or out += alpha * stencil
template <int MODE>
__global__ void k_pass2T(Tables T, const double* lam, const double* u, const double* aux, const double* t,
                         double alpha, int accumulate, double* out) {
  const int ng = T.ng;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
    double o[4];
    pass2T_cell<MODE>(T, i, lam, u, aux, t, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const size_t e = (size_t)c * ng + i;
      out[e] = accumulate ? fma(alpha, o[c], out[e]) : alpha * o[c];
    }
  }
}

// Conservation diagnostics: per block, in a fixed order, the sums of
// A_i h_i, A_i h_i (|u_i|^2/2 + g h_i/2) and A_i (zeta_i + f_i)^2 / (2 h_i).
constexpr int DIAG_THREADS = 256;
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(Tables T, const double* __restrict__ u, double* part) {
  __shared__ double red[3][DIAG_THREADS / 32];
  const int ng = T.ng;
  double m = 0.0, e = 0.0, z = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
    int nb[SLOTS];
    load_nbr(T, i, nb);
    double vor = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) vor = fma(ldtab(T.vd + (size_t)c * ng + i), u[(size_t)c * ng + i], vor);
#pragma unroll
    for (int k = 0; k < SLOTS; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        vor = fma(ldtab(T.vc + ((size_t)c * SLOTS + k) * ng + i), u[(size_t)c * ng + nb[k]], vor);
    const double eta = fma(T.two_omega, ldtab(T.nrm + 2 * (size_t)ng + i), vor);
    const double u0 = u[i], u1 = u[(size_t)ng + i], u2 = u[2 * (size_t)ng + i], h = u[3 * (size_t)ng + i];
    const double A = T.area[i];
    m = fma(A, h, m);
    e = fma(A * h, fma(0.5, fma(u0, u0, fma(u1, u1, u2 * u2)), 0.5 * T.g * h), e);
    z = fma(A, eta * eta / (2.0 * h), z);
  }
  double v[3] = {m, e, z};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0) red[k][warp] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < DIAG_THREADS / 32; ++w) s += red[threadIdx.x][w];
    part[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

// Sum of the block partials in block order (one thread per quantity).
__global__ void k_diag_sum(const double* part, int nblocks, double* out) {
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * 3 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

struct Comb {
  const double* x[6];
  double c[6];
  int k;
};

// out = sum_k c_k x_k over n elements
__global__ void k_lincomb(size_t n, Comb cb, double* out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < cb.k; ++k) s = fma(cb.c[k], cb.x[k][e], s);
    out[e] = s;
  }
}

__global__ void k_d2f(size_t n, const double* __restrict__ x, float* y) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}
__global__ void k_f2d(size_t n, const float* __restrict__ x, double* y) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = (double)x[e];
}

int grid_blocks(size_t work) {
  size_t b = (work + TPB - 1) / TPB;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

cudaEvent_t prof_event(const swe_grid* gc) {
  swe_grid* g = const_cast<swe_grid*>(gc);
  if (g->ev_used == g->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g->ev_pool.push_back(e);
  }
  return g->ev_pool[g->ev_used++];
}

void count_launches(const swe_grid* gc, int k) {
  swe_grid* g = const_cast<swe_grid*>(gc);
  if (g->prof_on) g->kernel_launches += k;
}

// Records a start event when profiling; finish() records the end and keeps the pair.
struct ProfSpan {
  swe_grid* g;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* list;
  ProfSpan(swe_grid* g_, cudaStream_t st_, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* l)
      : g(g_), st(st_), list(l) {
    if (g->prof_on && (a = prof_event(g))) cudaEventRecord(a, st);
  }
  void finish() {
    if (!a) return;
    cudaEvent_t b = prof_event(g);
    if (!b) return;
    cudaEventRecord(b, st);
    list->push_back({a, b});
    a = nullptr;
  }
};

int run_rhs(const swe_grid* g, const double* u, double* f, double alpha, cudaStream_t st) {
  const Tables& T = g->T;
  int nb = grid_blocks(T.ng);
  k_pass1<MODE_F><<<nb, TPB, 0, st>>>(T, u, 1.0, nullptr, g->tmp2);
  k_pass2<MODE_F><<<nb, TPB, 0, st>>>(T, u, 1.0, g->tmp2, nullptr, alpha, f);
  CK(cudaGetLastError());
  count_launches(g, 2);
  return SWE_OK;
}

int run_quad(const swe_grid* g, const double* d, double* out, double alpha, cudaStream_t st) {
  const Tables& T = g->T;
  int nb = grid_blocks(T.ng);
  k_pass1<MODE_Q><<<nb, TPB, 0, st>>>(T, d, 1.0, nullptr, g->tmp2);
  k_pass2<MODE_Q><<<nb, TPB, 0, st>>>(T, d, 1.0, g->tmp2, nullptr, alpha, out);
  CK(cudaGetLastError());
  count_launches(g, 2);
  return SWE_OK;
}

int run_lincomb(const swe_grid* g, double* out, std::initializer_list<std::pair<double, const double*>> terms,
                cudaStream_t st) {
  Comb cb{};
  cb.k = 0;
  for (auto& t : terms) {
    if (cb.k == 6) return fail(SWE_ERR_INVALID_ARG, "lincomb: too many terms");
    cb.c[cb.k] = t.first;
    cb.x[cb.k] = t.second;
    cb.k++;
  }
  size_t n = (size_t)4 * g->T.ng;
  k_lincomb<<<grid_blocks(n), TPB, 0, st>>>(n, cb, out);
  CK(cudaGetLastError());
  count_launches(g, 1);
  return SWE_OK;
}

// Thread 0 waits, with the poll of every grid barrier, for a flag that nothing
// sets; the wait ends at the time limit (or at once on a set abort word) and
// the kernel returns normally with the reason in s->abort.
__global__ void k_selftest_wait(GridSync* s, const int* flag, unsigned long long limit_ns) {
  if (threadIdx.x != 0) return;
  const volatile int* f = flag;
  bounded_spin(s, SWE_ERR_TIMEOUT, [&] { return *f == 0; }, limit_ns);
}

// -nu wl and -nu wld: the Laplacian weights of the dissipation -nu L (L x)
// (Eq. eq:swdis), so that pass 2 adds it with one FMA per term.
static void scaled_laplacian(const HostGrid& h, double nu, std::vector<double>& nwl, std::vector<double>& nwld) {
  nwl.resize(h.wl.size());
  nwld.resize(h.wld.size());
  for (size_t k = 0; k < nwl.size(); ++k) nwl[k] = -nu * h.wl[k];
  for (size_t k = 0; k < nwld.size(); ++k) nwld[k] = -nu * h.wld[k];
}

int upload_grid(swe_grid* g) {
  HostGrid& h = g->host;
  const size_t ng = h.ng;
  struct Part {
    const void* src;
    size_t bytes;
    void** dst;
  };
  const int32_t* d_nbr = nullptr;
  const double *d_nrm = nullptr, *d_wl = nullptr, *d_wld = nullptr, *d_nc = nullptr, *d_ndd = nullptr,
               *d_sdg = nullptr, *d_vc = nullptr, *d_vd = nullptr, *d_wlT = nullptr, *d_ncT = nullptr,
               *d_vcT = nullptr, *d_area = nullptr, *d_nwl = nullptr, *d_nwld = nullptr;
  // the kernels read the G diagonal ndd - sdg directly (table "sdg" of the
  // device copy holds that difference), and the dissipation's Laplacian
  // weights with -nu folded in
  std::vector<double> gdg(h.sdg.size());
  for (size_t k = 0; k < gdg.size(); ++k) gdg[k] = h.ndd[k] - h.sdg[k];
  std::vector<double> nwl, nwld;
  scaled_laplacian(h, g->T.nu, nwl, nwld);
  Part parts[] = {
      {h.nbr.data(), h.nbr.size() * 4, (void**)&d_nbr},  {h.xyz.data(), h.xyz.size() * 8, (void**)&d_nrm},
      {h.wl.data(), h.wl.size() * 8, (void**)&d_wl},     {h.wld.data(), h.wld.size() * 8, (void**)&d_wld},
      {h.nc.data(), h.nc.size() * 8, (void**)&d_nc},     {h.ndd.data(), h.ndd.size() * 8, (void**)&d_ndd},
      {gdg.data(), gdg.size() * 8, (void**)&d_sdg},  {h.vc.data(), h.vc.size() * 8, (void**)&d_vc},
      {h.vd.data(), h.vd.size() * 8, (void**)&d_vd},     {h.wlT.data(), h.wlT.size() * 8, (void**)&d_wlT},
      {h.ncT.data(), h.ncT.size() * 8, (void**)&d_ncT},  {h.vcT.data(), h.vcT.size() * 8, (void**)&d_vcT},
      {h.area.data(), h.area.size() * 8, (void**)&d_area},
      {nwl.data(), nwl.size() * 8, (void**)&d_nwl},      {nwld.data(), nwld.size() * 8, (void**)&d_nwld},
  };
  size_t total = 0;
  for (auto& p : parts) total += (p.bytes + 255) & ~size_t(255);
  CK(cudaMalloc(&g->dtab, total));
  g->tab_bytes = total;
  size_t off = 0;
  for (auto& p : parts) {
    char* dst = (char*)g->dtab + off;
    CK(cudaMemcpy(dst, p.src, p.bytes, cudaMemcpyHostToDevice));
    *p.dst = dst;
    off += (p.bytes + 255) & ~size_t(255);
  }
  (void)ng;
  Tables& T = g->T;
  T.nbr = d_nbr;
  T.nrm = d_nrm;
  T.wl = d_wl;
  T.wld = d_wld;
  T.nc = d_nc;
  T.ndd = d_ndd;
  T.gdg = d_sdg;
  T.vc = d_vc;
  T.vd = d_vd;
  T.wlT = d_wlT;
  T.ncT = d_ncT;
  T.vcT = d_vcT;
  T.area = d_area;
  T.nwl = d_nwl;
  T.nwld = d_nwld;
  return SWE_OK;
}

int ensure_workspace(swe_grid* g) {
  if (!g->dtab) return fail(SWE_ERR_INVALID_ARG, "grid was built on the host only");
  if (g->dws) return SWE_OK;
  if (phi_select(g->T.ng, 0, &g->launch) != 0 || phi_select(g->T.ng, 1, &g->launchF) != 0)
    return fail(SWE_ERR_CUDA, "occupancy query for phi kernel failed");
  const int nb = g->launch.nblocks;
  const size_t ng = g->T.ng, n = 4 * ng;
  size_t sizes[] = {
      (size_t)(KMAX + 1) * n * 8,  // Vbuf
      (size_t)(PMAX + 1) * n * 8,  // W
      8 * ng * 8,                  // tmp
      8 * ng * 8,                  // tmp2
      3 * n * 8,                   // Lring
      n * 8,                       // Zbuf
      4 * ng * 8,                  // aux
      (size_t)(nb > g->launchF.nblocks ? nb : g->launchF.nblocks) * NRED * 8,  // part
      (size_t)STAGE_VECS * n * 8,  // stage
      sizeof(PhiCtrl), sizeof(GridSync), sizeof(DevStats), (size_t)TRACE_CAP * sizeof(DevAttempt),
      sizeof(DevProfile)};
  size_t total = 0;
  for (size_t s : sizes) total += (s + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&g->dws, total);
  if (e != cudaSuccess) {
    g->dws = nullptr;
    return fail(SWE_ERR_NOMEM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
  }
  char* p = (char*)g->dws;
  void** dst[] = {(void**)&g->Vbuf,  (void**)&g->W,     (void**)&g->tmp,   (void**)&g->tmp2,
                  (void**)&g->Lring, (void**)&g->Zbuf,  (void**)&g->aux,   (void**)&g->part,
                  (void**)&g->stage, (void**)&g->ctrl,  (void**)&g->sync,  (void**)&g->stats,
                  (void**)&g->trace, (void**)&g->dprof};
  static_assert(sizeof(sizes) / sizeof(sizes[0]) == 14, "workspace layout");
  for (int k = 0; k < 14; ++k) {
    *dst[k] = p;
    p += (sizes[k] + 255) & ~size_t(255);
  }
  g->ws_bytes = total;
  CK(cudaMemset(g->dws, 0, total));
  return SWE_OK;
}

// FP32 copies of the operator tables and the FP32 workspace of the mixed path.
int ensure_mixed(swe_grid* g) {
  if (g->dwsF) return SWE_OK;
  const HostGrid& h = g->host;
  const size_t ng = h.ng, n = 4 * ng;
  std::vector<float> f;
  auto conv = [&](const std::vector<double>& src) {
    f.resize(src.size());
    for (size_t k = 0; k < src.size(); ++k) f[k] = (float)src[k];
  };
  struct Part {
    const std::vector<double>* src;
    const float* __restrict__* dst;
  };
  std::vector<double> gdg(h.sdg.size());
  for (size_t k = 0; k < gdg.size(); ++k) gdg[k] = h.ndd[k] - h.sdg[k];
  std::vector<double> nwl, nwld;
  scaled_laplacian(h, g->T.nu, nwl, nwld);
  TablesF& T = g->TF;
  Part parts[] = {{&h.xyz, &T.nrm}, {&h.wl, &T.wl},   {&h.wld, &T.wld}, {&h.nc, &T.nc},
                  {&h.ndd, &T.ndd}, {&gdg, &T.gdg},   {&h.vc, &T.vc},   {&h.vd, &T.vd},
                  {&nwl, &T.nwl},   {&nwld, &T.nwld}};
  size_t total = 0;
  for (auto& p : parts) total += (p.src->size() * 4 + 255) & ~size_t(255);
  CK(cudaMalloc(&g->dtabF, total));
  size_t off = 0;
  for (auto& p : parts) {
    conv(*p.src);
    char* dst = (char*)g->dtabF + off;
    CK(cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    *p.dst = (const float*)dst;
    off += (p.src->size() * 4 + 255) & ~size_t(255);
  }
  T.ng = (int)ng;
  T.nbr = g->T.nbr;
  T.nu = (float)g->T.nu;
  T.g = (float)g->T.g;
  T.two_omega = (float)g->T.two_omega;
  size_t sizes[] = {(size_t)(KMAX + 1) * n, (size_t)(PMAX + 1) * n, 8 * ng, 3 * n, n, 4 * ng, 4 * ng,
                    (size_t)(PMAX + 1) * n, (size_t)NSMAX * n};
  float** dst[] = {&g->VbufF, &g->WF, &g->tmpF, &g->LringF, &g->ZbufF, &g->auxF, &g->ulinF, &g->vinF, &g->youtF};
  size_t tot = 0;
  for (size_t s : sizes) tot += (s * 4 + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&g->dwsF, tot);
  if (e != cudaSuccess) {
    g->dwsF = nullptr;
    return fail(SWE_ERR_NOMEM, std::string("mixed workspace allocation failed: ") + cudaGetErrorString(e));
  }
  char* p = (char*)g->dwsF;
  for (int k = 0; k < 9; ++k) {
    *dst[k] = (float*)p;
    p += (sizes[k] * 4 + 255) & ~size_t(255);
  }
  CK(cudaMemset(g->dwsF, 0, tot));
  return SWE_OK;
}

int resolve_opts(const phi_opts* in, phi_opts& o) {
  if (in)
    o = *in;
  else
    swe_phi_opts_default(&o);
  if (!(o.tol > 0.0) || o.m_init < 1 || o.m_max < 1 || o.m_max > KMAX ||
      !(o.delta > 0.0) || !(o.gamma > 0.0) || !(o.kappa > 1.0) || o.max_reject < 0 || o.max_substeps < 1 ||
      o.iom < 2 || o.iom > KMAX ||
      (o.tol_mode != 0 && o.tol_mode != 1) || (o.replay && o.n_replay < 1) ||
      (o.precision != 0 && o.precision != 1))
    return fail(SWE_ERR_INVALID_ARG, "invalid phi_opts (m_max <= 64, 2 <= iom <= 64, tol > 0, kappa > 1)");
  return SWE_OK;
}

// Offsets of each call's records in a step's replay array: the landing rule
// of Algorithm 1 (R9 of the oracle) run over the records, call by call, with
// the outputs rho of each call.
int replay_split(const double* rec, int nrec, const std::vector<std::vector<double>>& rhos,
                 std::vector<int>& offs) {
  int pos = 0;
  for (size_t c = 0; c < rhos.size(); ++c) {
    offs[c] = pos;
    double t = 0.0;
    for (double rho : rhos[c]) {
      while (t < rho) {
        if (pos >= nrec) return fail(SWE_ERR_INVALID_ARG, "replay: too few records for the scheme's calls");
        const double tau = rec[3 * pos];
        const bool acc = rec[3 * pos + 2] != 0.0;
        ++pos;
        if (!(tau > 0.0)) return fail(SWE_ERR_INVALID_ARG, "replay: non-positive step size");
        const double remaining = rho - t;
        const bool land = tau >= remaining * (1.0 - 1e-12);
        if (acc) t = land ? rho : t + tau;
      }
    }
  }
  return SWE_OK;
}

int stage_replay(swe_grid* g, const phi_opts& o, cudaStream_t st) {
  if (!o.replay) return SWE_OK;
  if (o.n_replay > g->replay_cap) {
    if (g->replay) cudaFree(g->replay);
    g->replay = nullptr;
    CK(cudaMalloc(&g->replay, (size_t)o.n_replay * 3 * sizeof(double)));
    g->replay_cap = o.n_replay;
  }
  CK(cudaMemcpyAsync(g->replay, o.replay, (size_t)o.n_replay * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
  return SWE_OK;
}

// One phipm_simul_iom2 evaluation; aux of u_lin must already be in g->aux.
template <class A>
void fill_phi_args(swe_grid* g, A& a, double dt, int p, int ns, const double* rho, const phi_opts& o,
                   int call_index, int* m_slot, int replay_offset) {
  a.dt = dt;
  a.p = p;
  a.ns = ns;
  for (int i = 0; i < ns; ++i) a.rho[i] = rho[i];
  a.part = g->part;
  a.ctrl = g->ctrl;
  a.sync = g->sync;
  a.stats = g->stats;
  a.trace = g->trace;
  a.trace_cap = TRACE_CAP;
  a.call_index = call_index;
  a.m_slot = m_slot;
  a.replay = o.replay ? g->replay + 3 * (size_t)replay_offset : nullptr;
  a.n_replay = o.replay ? o.n_replay - replay_offset : 0;
  a.tol = o.tol;
  a.delta = o.delta;
  a.gamma = o.gamma;
  a.kappa = o.kappa;
  a.tol_mode = o.tol_mode;
  a.m_init = o.m_init;
  a.m_max = o.m_max;
  a.max_reject = o.max_reject;
  a.max_substeps = o.max_substeps;
  a.iom = o.iom;
  a.nA = g->host.nA;
  a.prof = g->prof_on ? g->dprof : nullptr;
}

// Linearisation data of u_lin for the following phi calls: eta and n x u
// (and, in the mixed path, the FP32 copy of u_lin).
int prepare_lin(swe_grid* g, const double* u_lin, const phi_opts& o, cudaStream_t st) {
  const int nb = grid_blocks(g->T.ng);
  if (o.precision == 0) {
    k_aux<double><<<nb, TPB, 0, st>>>(g->T, u_lin, g->aux);
    CK(cudaGetLastError());
    count_launches(g, 1);
    return SWE_OK;
  }
  const size_t n = (size_t)4 * g->T.ng;
  k_d2f<<<grid_blocks(n), TPB, 0, st>>>(n, u_lin, g->ulinF);
  k_aux<float><<<nb, TPB, 0, st>>>(g->TF, g->ulinF, g->auxF);
  CK(cudaGetLastError());
  count_launches(g, 2);
  return SWE_OK;
}

// One phipm_simul_iom2 evaluation; prepare_lin(u_lin) must precede it on the stream.
// Buffers of the wide-window path (iom > 2) for precision R: (KMAX + 1)
// Laplacian planes and nblocks x WIDE_STRIDE partial sums.
template <typename R>
int ensure_wide(swe_grid* g, R** Lbuf, double** partw) {
  void*& mem = sizeof(R) == 8 ? g->dwide : g->dwideF;
  const PhiLaunch& L = sizeof(R) == 8 ? g->launch : g->launchF;
  const size_t n = (size_t)4 * g->T.ng;
  const size_t lbytes = ((size_t)(KMAX + 1) * n * sizeof(R) + 255) & ~size_t(255);
  if (!mem) {
    const size_t total = lbytes + (size_t)L.nblocks * WIDE_STRIDE * sizeof(double);
    cudaError_t e = cudaMalloc(&mem, total);
    if (e != cudaSuccess) {
      mem = nullptr;
      return fail(SWE_ERR_NOMEM, std::string("wide-window buffers: ") + cudaGetErrorString(e));
    }
  }
  *Lbuf = (R*)mem;
  *partw = (double*)((char*)mem + lbytes);
  return SWE_OK;
}

// Tape of one recorded call (device pointers inside swe_grid::dtape).
struct TapeCall {
  double* W = nullptr;
  double* V = nullptr;
  long long* offV = nullptr;  // K offsets, then K basis-slot counts (as long long)
  TapeSub* sub = nullptr;
  int K = 0;  // accepted substeps
  int p = 0;
};

int phi_call(swe_grid* g, const double* u_lin, double dt, int p, const double* const* v, int ns,
             const double* rho, double* const* y_out, const phi_opts& o, int call_index, int* m_slot,
             int replay_offset, cudaStream_t st, const TapeCall* tape = nullptr) {
  CK(cudaMemsetAsync(g->sync, 0, sizeof(GridSync), st));
  if (o.precision == 0) {
    PhiArgs a{};
    a.T = g->T;
    a.u_lin = u_lin;
    a.aux = g->aux;
    for (int i = 0; i < ns; ++i) a.y_out[i] = y_out[i];
    for (int l = 0; l <= p; ++l) a.v[l] = v[l];
    a.Vbuf = g->Vbuf;
    a.W = g->W;
    a.tmp = g->tmp;
    a.Lring = g->Lring;
    a.Zbuf = g->Zbuf;
    fill_phi_args(g, a, dt, p, ns, rho, o, call_index, m_slot, replay_offset);
    if (o.iom > 2) {
      int rc = ensure_wide<double>(g, &a.Lbuf, &a.partw);
      if (rc) return rc;
    }
    if (tape) {
      a.tapeW = tape->W;
      a.tapeV = tape->V;
      a.tape_offV = tape->offV;
      a.tape_sub = tape->sub;
      a.tape_cap = tape->K;
    }
    ProfSpan span(g, st, &g->phi_ev);
    int e = launch_phi_kernel(g->launch, a, st);
    if (e != 0) return cuda_fail((cudaError_t)e, "cudaLaunchCooperativeKernel(phi_kernel)");
    span.finish();
    count_launches(g, 1);
    return SWE_OK;
  }
  // mixed precision: FP32 copies of the inputs, FP32 outputs widened afterwards
  const size_t n = (size_t)4 * g->T.ng;
  PhiArgsF a{};
  a.T = g->TF;
  a.u_lin = g->ulinF;
  a.aux = g->auxF;
  for (int l = 0; l <= p; ++l) {
    if (v[l]) {
      k_d2f<<<grid_blocks(n), TPB, 0, st>>>(n, v[l], g->vinF + (size_t)l * n);
      count_launches(g, 1);
      a.v[l] = g->vinF + (size_t)l * n;
    } else {
      a.v[l] = nullptr;
    }
  }
  for (int i = 0; i < ns; ++i) a.y_out[i] = g->youtF + (size_t)i * n;
  a.Vbuf = g->VbufF;
  a.W = g->WF;
  a.tmp = g->tmpF;
  a.Lring = g->LringF;
  a.Zbuf = g->ZbufF;
  fill_phi_args(g, a, dt, p, ns, rho, o, call_index, m_slot, replay_offset);
  if (o.iom > 2) {
    int rc = ensure_wide<float>(g, &a.Lbuf, &a.partw);
    if (rc) return rc;
  }
  ProfSpan span(g, st, &g->phi_ev);
  int e = launch_phi_kernel(g->launchF, a, st);
  if (e != 0) return cuda_fail((cudaError_t)e, "cudaLaunchCooperativeKernel(phi_kernel<float>)");
  span.finish();
  count_launches(g, 1);
  for (int i = 0; i < ns; ++i) {
    k_f2d<<<grid_blocks(n), TPB, 0, st>>>(n, g->youtF + (size_t)i * n, y_out[i]);
    count_launches(g, 1);
  }
  CK(cudaGetLastError());
  return SWE_OK;
}

int validate_phi_args(int p, const double* const* v, int ns, const double* rho, double* const* y_out) {
  if (p < 1 || p > PMAX) return fail(SWE_ERR_INVALID_ARG, "p must be in [1, 4]");
  if (ns < 1 || ns > NSMAX) return fail(SWE_ERR_INVALID_ARG, "ns must be in [1, 8]");
  if (!v || !rho || !y_out) return fail(SWE_ERR_INVALID_ARG, "v, rho and y_out are required");
  if (!(rho[0] > 0.0) || !(rho[ns - 1] <= 1.0)) return fail(SWE_ERR_INVALID_ARG, "rho must lie in (0, 1]");
  for (int i = 1; i < ns; ++i)
    if (!(rho[i] > rho[i - 1])) return fail(SWE_ERR_INVALID_ARG, "rho must be increasing");
  for (int i = 0; i < ns; ++i)
    if (!y_out[i]) return fail(SWE_ERR_INVALID_ARG, "y_out entries must be non-NULL");
  return SWE_OK;
}

int read_stats(swe_grid* g, phi_stats* stats, cudaStream_t st) {
  if (!stats) return SWE_OK;
  DevStats ds;
  CK(cudaMemcpyAsync(&ds, g->stats, sizeof(DevStats), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  stats->n_jv = ds.n_jv;
  stats->n_substeps = ds.n_sub;
  stats->n_reject = ds.n_rej;
  stats->m_last = ds.m_last;
  stats->m_max_used = ds.m_max_used;
  stats->status = ds.status;
  int nt = ds.n_trace < TRACE_CAP ? ds.n_trace : TRACE_CAP;
  stats->n_trace = 0;
  if (stats->trace && stats->trace_cap > 0) {
    int k = nt < stats->trace_cap ? nt : stats->trace_cap;
    if (k > 0) {
      static_assert(sizeof(DevAttempt) == sizeof(phi_attempt), "trace record layout");
      CK(cudaMemcpy(stats->trace, g->trace, (size_t)k * sizeof(DevAttempt), cudaMemcpyDeviceToHost));
    }
    stats->n_trace = k;
  }
  return SWE_OK;
}

// ---------------------------------------------------------------------------
// adjoint of a step (exprb_step_adjoint)
// ---------------------------------------------------------------------------
constexpr int ADJ_XS_STEPS = 4096;  // scaling steps of one exponential the scratch holds
constexpr int ADJ_VECS = 16;        // scheme-level vectors of the adjoint driver

int ensure_adjoint(swe_grid* g) {
  if (g->dadj) return SWE_OK;
  int nb = 0, thr = 0;
  if (adj_max_blocks(&nb, &thr) != 0) return fail(SWE_ERR_CUDA, "occupancy query for adj_kernel failed");
  const size_t ng = g->T.ng, n = 4 * ng;
  const size_t mw = KMAX + PMAX + 2;
  size_t sizes[] = {n * 8,                                      // Y
                    (size_t)(PMAX + 1) * n * 8,                 // Wb
                    2 * n * 8,                                  // X
                    2 * n * 8,                                  // P
                    10 * ng * 8,                                // PL
                    n * 8,                                      // Zb
                    (size_t)nb * NRED * 8,                      // part
                    (size_t)nb * ADJ_KW * 8,                    // partw
                    (size_t)(ADJ_XS_STEPS + 40) * mw * 8,       // xs
                    (size_t)ADJ_VECS * n * 8,                   // scheme vectors
                    sizeof(AdjCtrl), sizeof(int)};
  void** dst[] = {(void**)&g->aY,   (void**)&g->aWb,    (void**)&g->aX,  (void**)&g->aP,
                  (void**)&g->aPL,  (void**)&g->aZb,    (void**)&g->apart, (void**)&g->apartw,
                  (void**)&g->axs,  (void**)&g->avec,   (void**)&g->actrl, (void**)&g->adj_status};
  constexpr int NP = sizeof(sizes) / sizeof(sizes[0]);
  static_assert(NP == 12, "adjoint workspace layout");
  size_t total = 0;
  for (size_t x : sizes) total += (x + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&g->dadj, total);
  if (e != cudaSuccess) {
    g->dadj = nullptr;
    return fail(SWE_ERR_NOMEM, std::string("adjoint workspace allocation failed: ") + cudaGetErrorString(e));
  }
  char* q = (char*)g->dadj;
  for (int k = 0; k < NP; ++k) {
    *dst[k] = q;
    q += (sizes[k] + 255) & ~size_t(255);
  }
  g->adj_nblocks = nb;
  CK(cudaMemset(g->dadj, 0, total));
  CK(cudaEventCreateWithFlags(&g->stage_ev, cudaEventDisableTiming));
  return SWE_OK;
}

// Splits a step's trace into calls and lays the tapes out: per call, the
// accepted substeps and, per substep, the largest Krylov size of its
// attempts (the basis the replay builds).  Fills `replay` with the calls'
// (tau, m, accepted) records in call order and `first` with each call's
// offset into it.
struct TapePlan {
  std::vector<double> replay;
  std::vector<int> first, count;
  std::vector<std::vector<int>> mmax;  // per call, per accepted substep
};

int plan_tape(const phi_attempt* trace, int n_trace, int ncalls, TapePlan& P) {
  P.first.assign(ncalls, 0);
  P.count.assign(ncalls, 0);
  P.mmax.assign(ncalls, {});
  P.replay.clear();
  int pos = 0;
  for (int c = 0; c < ncalls; ++c) {
    P.first[c] = (int)(P.replay.size() / 3);
    int cur = 0;
    bool open = false;
    while (pos < n_trace && trace[pos].call == c) {
      const phi_attempt& r = trace[pos++];
      if (r.m < 1 || r.m > KMAX || !(r.tau > 0.0)) return fail(SWE_ERR_INVALID_ARG, "trace: invalid attempt");
      P.replay.push_back(r.tau);
      P.replay.push_back((double)r.m);
      P.replay.push_back(r.accepted ? 1.0 : 0.0);
      cur = std::max(cur, r.m);
      open = true;
      if (r.accepted) {
        P.mmax[c].push_back(cur);
        cur = 0;
        open = false;
      }
    }
    P.count[c] = (int)(P.replay.size() / 3) - P.first[c];
    if (open) return fail(SWE_ERR_INVALID_ARG, "trace: a call ends with a rejected attempt");
    if (P.mmax[c].empty()) return fail(SWE_ERR_INVALID_ARG, "trace: a call has no accepted substep");
  }
  if (pos != n_trace) return fail(SWE_ERR_INVALID_ARG, "trace: call indices do not match the scheme");
  return SWE_OK;
}

int alloc_tapes(swe_grid* g, const TapePlan& P, const int* pc, int ncalls, TapeCall* out, cudaStream_t st) {
  const size_t n = (size_t)4 * g->T.ng;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t total = 0, nstage = 0;
  std::vector<size_t> offW(ncalls), offV(ncalls), offO(ncalls), offS(ncalls);
  for (int c = 0; c < ncalls; ++c) {
    const size_t K = P.mmax[c].size();
    size_t vsz = 0;
    for (int m : P.mmax[c]) vsz += (size_t)(m + 1) * n;
    offW[c] = total;
    total += al((K + 1) * (size_t)(pc[c] + 1) * n * 8);
    offV[c] = total;
    total += al(vsz * 8);
    offO[c] = total;
    total += al(2 * K * sizeof(long long));
    offS[c] = total;
    total += al(K * sizeof(TapeSub));
    nstage += 2 * K;
  }
  if (total > g->tape_bytes) {
    if (g->dtape) {
      CK(cudaStreamSynchronize(st));
      cudaFree(g->dtape);
    }
    g->dtape = nullptr;
    g->tape_bytes = 0;
    cudaError_t e = cudaMalloc(&g->dtape, total);
    if (e != cudaSuccess) {
      g->dtape = nullptr;
      return fail(SWE_ERR_NOMEM, std::string("tape allocation failed: ") + cudaGetErrorString(e));
    }
    g->tape_bytes = total;
  }
  // the previous step's layout copies must have left the pinned staging
  CK(cudaEventSynchronize(g->stage_ev));
  if (nstage > g->hstage_cap) {
    if (g->hstage) cudaFreeHost(g->hstage);
    g->hstage = nullptr;
    g->hstage_cap = 0;
    CK(cudaMallocHost(&g->hstage, nstage * sizeof(long long)));
    g->hstage_cap = nstage;
  }
  char* base = (char*)g->dtape;
  size_t pos = 0;
  for (int c = 0; c < ncalls; ++c) {
    TapeCall& t = out[c];
    t.W = (double*)(base + offW[c]);
    t.V = (double*)(base + offV[c]);
    t.offV = (long long*)(base + offO[c]);
    t.sub = (TapeSub*)(base + offS[c]);
    t.K = (int)P.mmax[c].size();
    t.p = pc[c];
    long long* h = g->hstage + pos;
    long long acc = 0;
    for (int k = 0; k < t.K; ++k) {
      h[k] = acc;
      h[t.K + k] = P.mmax[c][k];
      acc += (long long)(P.mmax[c][k] + 1) * (long long)n;
    }
    CK(cudaMemcpyAsync(t.offV, h, 2 * (size_t)t.K * sizeof(long long), cudaMemcpyHostToDevice, st));
    pos += 2 * (size_t)t.K;
  }
  CK(cudaEventRecord(g->stage_ev, st));
  return SWE_OK;
}

// Reverse of one recorded call: vbar[l] += ..., ubar += ...
int adj_call(swe_grid* g, const TapeCall& tp, const double* u_lin, double dt, const double* const* ybar,
             int ns, double* const* vbar, double* ubar, cudaStream_t st) {
  CK(cudaMemsetAsync(g->sync, 0, sizeof(GridSync), st));
  CK(cudaMemsetAsync(g->actrl, 0, sizeof(AdjCtrl), st));
  AdjArgs a{};
  a.T = g->T;
  a.u_lin = u_lin;
  a.aux = g->aux;
  a.dt = dt;
  a.p = tp.p;
  a.nsub = tp.K;
  for (int i = 0; i < ns; ++i) a.ybar[i] = ybar[i];
  for (int l = 0; l <= tp.p; ++l) a.vbar[l] = vbar[l];
  a.ubar = ubar;
  a.tapeW = tp.W;
  a.tapeV = tp.V;
  a.tape_offV = tp.offV;
  a.tape_mmax = tp.offV + tp.K;
  a.tape_sub = tp.sub;
  a.ns = ns;
  a.status_out = g->adj_status;
  a.Y = g->aY;
  a.Wb = g->aWb;
  a.X = g->aX;
  a.P = g->aP;
  a.PL = g->aPL;
  a.Zb = g->aZb;
  a.part = g->apart;
  a.partw = g->apartw;
  a.xs = g->axs;
  a.xs_steps = ADJ_XS_STEPS;
  a.ctrl = g->actrl;
  a.sync = g->sync;
  a.prof = nullptr;
  int e = launch_adj_kernel(a, g->adj_nblocks, st);
  if (e != 0) return cuda_fail((cudaError_t)e, "cudaLaunchCooperativeKernel(adj_kernel)");
  count_launches(g, 1);
  return SWE_OK;
}

// out = (accumulate ? out : 0) + alpha * J(u)^T lam (MODE_JT, aux of u in
// g->aux) or alpha * (J(x) - J(0))^T lam (MODE_QT, aux of x written to auxq).
template <int MODE>
int run_transposed(swe_grid* g, const double* u, const double* lam, double alpha, int accumulate, double* out,
                   double* auxq, cudaStream_t st) {
  Tables T = g->T;
  const int nb = grid_blocks(T.ng);
  const double* aux = g->aux;
  if (MODE == MODE_QT) {
    T.two_omega = 0.0;
    k_aux<double><<<nb, TPB, 0, st>>>(T, u, auxq);
    count_launches(g, 1);
    aux = auxq;
  }
  k_pass1T<MODE><<<nb, TPB, 0, st>>>(T, lam, aux, g->tmp2);
  k_pass2T<MODE><<<nb, TPB, 0, st>>>(T, lam, u, aux, g->tmp2, alpha, accumulate, out);
  CK(cudaGetLastError());
  count_launches(g, 2);
  return SWE_OK;
}

}  // namespace

// Accessors for the allocation-free entry point (swe_noalloc.cu).
namespace swe {
int grid_device_tables(const swe_grid* g, Tables* out, int* device) {
  if (!g->dtab) return fail(SWE_ERR_INVALID_ARG, "grid was built on the host only");
  *out = g->T;
  *device = g->device;
  return SWE_OK;
}
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace swe

// ---------------------------------------------------------------------------
// public entry points
// ---------------------------------------------------------------------------
extern "C" {

void swe_phi_opts_default(phi_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->tol_mode = 0;
  o->m_init = 1;
  o->m_max = 64;
  o->iom = 2;
  o->delta = 1.4;
  o->gamma = 0.8;
  o->kappa = 2.0;
  o->max_reject = 200;
  o->max_substeps = 4096;
  o->m_carry = 1;
  o->replay = nullptr;
  o->n_replay = 0;
}

const char* swe_last_error(void) { return g_last_error.c_str(); }

static int create_grid(int level, double radius, double g, double omega, double gamma_h, int reorder,
                       bool device, swe_grid** out) {
  if (!out) return fail(SWE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!(radius > 0.0) || !(g > 0.0) || !(gamma_h >= 0.0) || !std::isfinite(omega))
    return fail(SWE_ERR_INVALID_ARG, "radius, g must be > 0 and gamma_h >= 0");
  swe_grid* G = new (std::nothrow) swe_grid();
  if (!G) return fail(SWE_ERR_NOMEM, "host allocation failed");
  const char* err = nullptr;
  if (build_host_grid(level, radius, reorder != 0, G->host, &err) != 0) {
    delete G;
    return fail(SWE_ERR_INVALID_ARG, err ? err : "grid construction failed");
  }
  const int ng = G->host.ng;
  double dx = std::sqrt(4.0 * M_PI * radius * radius / ng);
  G->T.ng = ng;
  G->T.nu = gamma_h * dx * dx * dx * dx / 240.0;  // Eq. eq:niu, n_gamma = 4, dt_e = 240 s
  G->T.g = g;
  G->T.two_omega = 2.0 * omega;
  if (!device) {
    *out = G;
    return SWE_OK;
  }
  cudaGetDevice(&G->device);
  int rc = upload_grid(G);
  if (rc != SWE_OK) {
    if (G->dtab) cudaFree(G->dtab);
    delete G;
    return rc;
  }
  *out = G;
  return SWE_OK;
}

int swe_create_grid(int level, double radius, double g, double omega, double gamma_h, int reorder,
                    swe_grid** out) {
  return create_grid(level, radius, g, omega, gamma_h, reorder, true, out);
}

int swe_create_grid_host(int level, double radius, double g, double omega, double gamma_h,
                         int reorder, swe_grid** out) {
  return create_grid(level, radius, g, omega, gamma_h, reorder, false, out);
}

int swe_grid_export(const swe_grid* g, const char* table, void* out, int64_t count) {
  if (!g || !table || !out) return fail(SWE_ERR_INVALID_ARG, "grid, table and out are required");
  const HostGrid& h = g->host;
  auto put = [&](const void* src, size_t elems, size_t esz) {
    if ((int64_t)elems != count) return fail(SWE_ERR_INVALID_ARG, std::string("count mismatch for ") + table);
    std::memcpy(out, src, elems * esz);
    return (int)SWE_OK;
  };
  std::string t(table);
  if (t == "nbr") return put(h.nbr.data(), h.nbr.size(), 4);
  if (t == "gen") return put(h.gen.data(), h.gen.size(), 4);
  if (t == "wl") return put(h.wl.data(), h.wl.size(), 8);
  if (t == "wld") return put(h.wld.data(), h.wld.size(), 8);
  if (t == "nc") return put(h.nc.data(), h.nc.size(), 8);
  if (t == "ndd") return put(h.ndd.data(), h.ndd.size(), 8);
  if (t == "sdg") return put(h.sdg.data(), h.sdg.size(), 8);
  if (t == "vc") return put(h.vc.data(), h.vc.size(), 8);
  if (t == "vd") return put(h.vd.data(), h.vd.size(), 8);
  if (t == "wlT") return put(h.wlT.data(), h.wlT.size(), 8);
  if (t == "ncT") return put(h.ncT.data(), h.ncT.size(), 8);
  if (t == "vcT") return put(h.vcT.data(), h.vcT.size(), 8);
  return fail(SWE_ERR_INVALID_ARG, std::string("unknown table ") + table);
}

void swe_destroy_grid(swe_grid* g) {
  if (!g) return;
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  if (g->dtab) cudaFree(g->dtab);
  if (g->dws) cudaFree(g->dws);
  if (g->dtabF) cudaFree(g->dtabF);
  if (g->dwsF) cudaFree(g->dwsF);
  if (g->replay) cudaFree(g->replay);
  if (g->dadj) cudaFree(g->dadj);
  if (g->dtape) cudaFree(g->dtape);
  if (g->hstage) cudaFreeHost(g->hstage);
  if (g->stage_ev) cudaEventDestroy(g->stage_ev);
  if (g->dhs) cudaFree(g->dhs);
  if (g->dwide) cudaFree(g->dwide);
  if (g->dwideF) cudaFree(g->dwideF);
  delete g;
}

int swe_grid_query(const swe_grid* g, int64_t* ncells, int64_t* n, int64_t* nA, double* nu) {
  if (!g) return fail(SWE_ERR_INVALID_ARG, "grid is NULL");
  if (ncells) *ncells = g->host.ng;
  if (n) *n = 4 * (int64_t)g->host.ng;
  if (nA) *nA = g->host.nA;
  if (nu) *nu = g->T.nu;
  return SWE_OK;
}

int swe_grid_cell_centres(const swe_grid* g, double* xyz) {
  if (!g || !xyz) return fail(SWE_ERR_INVALID_ARG, "grid and xyz are required");
  std::memcpy(xyz, g->host.xyz.data(), g->host.xyz.size() * sizeof(double));
  return SWE_OK;
}

int swe_grid_cell_areas(const swe_grid* g, double* area) {
  if (!g || !area) return fail(SWE_ERR_INVALID_ARG, "grid and area are required");
  std::memcpy(area, g->host.area.data(), g->host.area.size() * sizeof(double));
  return SWE_OK;
}

int swe_rhs(const swe_grid* gc, const double* u, double* f, void* stream) {
  swe_grid* g = const_cast<swe_grid*>(gc);
  if (!g || !u || !f) return fail(SWE_ERR_INVALID_ARG, "swe_rhs: NULL argument");
  int rc = ensure_workspace(g);
  if (rc) return rc;
  return run_rhs(g, u, f, 1.0, S(stream));
}

int swe_jv(const swe_grid* gc, const double* u, const double* x, double* jx, void* stream) {
  swe_grid* g = const_cast<swe_grid*>(gc);
  if (!g || !u || !x || !jx) return fail(SWE_ERR_INVALID_ARG, "swe_jv: NULL argument");
  int rc = ensure_workspace(g);
  if (rc) return rc;
  const Tables& T = g->T;
  cudaStream_t st = S(stream);
  int nb = grid_blocks(T.ng);
  k_aux<double><<<nb, TPB, 0, st>>>(T, u, g->aux);
  k_pass1<MODE_J><<<nb, TPB, 0, st>>>(T, x, 1.0, u, g->tmp2);
  k_pass2<MODE_J><<<nb, TPB, 0, st>>>(T, x, 1.0, g->tmp2, g->aux, 1.0, jx);
  CK(cudaGetLastError());
  count_launches(g, 3);
  return SWE_OK;
}

int swe_grid_set_topography(swe_grid* g, const double* hs_host) {
  if (!g) return fail(SWE_ERR_INVALID_ARG, "swe_grid_set_topography: NULL grid");
  if (!g->dtab) return fail(SWE_ERR_INVALID_ARG, "grid was built on the host only");
  CK(cudaDeviceSynchronize());  // no work in flight reads the old field
  if (!hs_host) {
    if (g->dhs) cudaFree(g->dhs);
    g->dhs = nullptr;
    g->T.hs = nullptr;
    return SWE_OK;
  }
  const size_t bytes = (size_t)g->T.ng * sizeof(double);
  if (!g->dhs) {
    cudaError_t e = cudaMalloc(&g->dhs, bytes);
    if (e != cudaSuccess) {
      g->dhs = nullptr;
      return fail(SWE_ERR_NOMEM, std::string("topography allocation failed: ") + cudaGetErrorString(e));
    }
  }
  CK(cudaMemcpy(g->dhs, hs_host, bytes, cudaMemcpyHostToDevice));
  g->T.hs = g->dhs;
  return SWE_OK;
}

int swe_diagnostics(const swe_grid* gc, const double* u, double* out_host, void* stream) {
  swe_grid* g = const_cast<swe_grid*>(gc);
  if (!g || !u || !out_host) return fail(SWE_ERR_INVALID_ARG, "swe_diagnostics: NULL argument");
  int rc = ensure_workspace(g);
  if (rc) return rc;
  cudaStream_t st = S(stream);
  const int nb = std::min(grid_blocks(g->T.ng), 4 * 152);
  double* part = g->tmp2;              // nb x 3 partials (tmp2 holds 8 ng doubles)
  double* res = g->tmp2 + (size_t)3 * nb;
  if ((size_t)3 * nb + 3 > (size_t)8 * g->T.ng) return fail(SWE_ERR_INVALID_ARG, "swe_diagnostics: grid too small");
  k_diag<<<nb, DIAG_THREADS, 0, st>>>(g->T, u, part);
  k_diag_sum<<<1, 32, 0, st>>>(part, nb, res);
  CK(cudaGetLastError());
  count_launches(g, 2);
  CK(cudaMemcpyAsync(out_host, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SWE_OK;
}

int swe_jtv(const swe_grid* gc, const double* u, const double* lam, double* out, void* stream) {
  swe_grid* g = const_cast<swe_grid*>(gc);
  if (!g || !u || !lam || !out) return fail(SWE_ERR_INVALID_ARG, "swe_jtv: NULL argument");
  if (lam == out) return fail(SWE_ERR_INVALID_ARG, "swe_jtv: lam and out must not alias");
  int rc = ensure_workspace(g);
  if (rc) return rc;
  const Tables& T = g->T;
  cudaStream_t st = S(stream);
  int nb = grid_blocks(T.ng);
  k_aux<double><<<nb, TPB, 0, st>>>(T, u, g->aux);
  k_pass1T<MODE_JT><<<nb, TPB, 0, st>>>(T, lam, g->aux, g->tmp2);
  k_pass2T<MODE_JT><<<nb, TPB, 0, st>>>(T, lam, u, g->aux, g->tmp2, 1.0, 0, out);
  CK(cudaGetLastError());
  count_launches(g, 3);
  return SWE_OK;
}

int swe_dqtv(const swe_grid* gc, const double* x, const double* lam, double* out, void* stream) {
  swe_grid* g = const_cast<swe_grid*>(gc);
  if (!g || !x || !lam || !out) return fail(SWE_ERR_INVALID_ARG, "swe_dqtv: NULL argument");
  if (lam == out) return fail(SWE_ERR_INVALID_ARG, "swe_dqtv: lam and out must not alias");
  int rc = ensure_workspace(g);
  if (rc) return rc;
  Tables T0 = g->T;
  T0.two_omega = 0.0;  // eta of x without the planetary vorticity
  cudaStream_t st = S(stream);
  int nb = grid_blocks(T0.ng);
  k_aux<double><<<nb, TPB, 0, st>>>(T0, x, g->aux);
  k_pass1T<MODE_QT><<<nb, TPB, 0, st>>>(T0, lam, g->aux, g->tmp2);
  k_pass2T<MODE_QT><<<nb, TPB, 0, st>>>(T0, lam, x, g->aux, g->tmp2, 1.0, 0, out);
  CK(cudaGetLastError());
  count_launches(g, 3);
  return SWE_OK;
}

int phi_action(swe_grid* g, const double* u_lin, double dt, int p, const double* const* v, int ns,
               const double* rho, double* const* y_out, const phi_opts* opts, phi_stats* stats,
               void* stream) {
  if (!g || !u_lin) return fail(SWE_ERR_INVALID_ARG, "phi_action: NULL grid or u_lin");
  int rc = validate_phi_args(p, v, ns, rho, y_out);
  if (rc) return rc;
  phi_opts o;
  if ((rc = resolve_opts(opts, o))) return rc;
  if ((rc = ensure_workspace(g))) return rc;
  cudaStream_t st = S(stream);
  if ((rc = stage_replay(g, o, st))) return rc;
  if (o.precision == 1 && (rc = ensure_mixed(g))) return rc;
  ProfSpan span(g, st, &g->call_ev);
  CK(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), st));
  if ((rc = prepare_lin(g, u_lin, o, st))) return rc;
  if ((rc = phi_call(g, u_lin, dt, p, v, ns, rho, y_out, o, 0, nullptr, 0, st))) return rc;
  span.finish();
  return read_stats(g, stats, st);
}

int swe_scheme_state_create(const swe_grid* g, swe_scheme_state** out) {
  if (!g || !out) return fail(SWE_ERR_INVALID_ARG, "grid and out are required");
  swe_scheme_state* s = new (std::nothrow) swe_scheme_state();
  if (!s) return fail(SWE_ERR_NOMEM, "host allocation failed");
  s->grid = g;
  size_t n = (size_t)4 * g->host.ng;
  cudaError_t e = cudaMalloc(&s->u_prev, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->m_slots, 8 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s->m_slots, 0, 8 * sizeof(int));
  if (e != cudaSuccess) {
    if (s->u_prev) cudaFree(s->u_prev);
    if (s->m_slots) cudaFree(s->m_slots);
    delete s;
    return fail(SWE_ERR_NOMEM, std::string("scheme state allocation: ") + cudaGetErrorString(e));
  }
  *out = s;
  return SWE_OK;
}

int swe_scheme_state_reset(swe_scheme_state* s) {
  if (!s) return fail(SWE_ERR_INVALID_ARG, "state is NULL");
  s->have_prev = 0;
  CK(cudaMemset(s->m_slots, 0, 8 * sizeof(int)));
  return SWE_OK;
}

void swe_scheme_state_destroy(swe_scheme_state* s) {
  if (!s) return;
  if (s->u_prev) cudaFree(s->u_prev);
  if (s->m_slots) cudaFree(s->m_slots);
  delete s;
}

int exprb_step(swe_grid* g, int scheme, double dt, const double* u_n, double* u_np1,
               swe_scheme_state* state, const phi_opts* opts, phi_stats* stats, void* stream) {
  if (!g || !u_n || !u_np1 || !state) return fail(SWE_ERR_INVALID_ARG, "exprb_step: NULL argument");
  if (state->grid != g) return fail(SWE_ERR_INVALID_ARG, "exprb_step: state belongs to another grid");
  if (u_n == u_np1) return fail(SWE_ERR_INVALID_ARG, "exprb_step: u_n and u_np1 must differ");
  if (scheme < SWE_EPI2 || scheme > SWE_EPI3) return fail(SWE_ERR_INVALID_ARG, "unknown scheme");
  int rc;
  phi_opts o;
  if ((rc = resolve_opts(opts, o))) return rc;
  if ((rc = ensure_workspace(g))) return rc;
  cudaStream_t st = S(stream);
  if ((rc = stage_replay(g, o, st))) return rc;
  const size_t n = (size_t)4 * g->T.ng;
  double* B[STAGE_VECS];
  for (int k = 0; k < STAGE_VECS; ++k) B[k] = g->stage + (size_t)k * n;
  double* vF = B[0];
  if (o.precision == 1 && (rc = ensure_mixed(g))) return rc;
  ProfSpan span(g, st, &g->call_ev);
  CK(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), st));
  if ((rc = prepare_lin(g, u_n, o, st))) return rc;
  if ((rc = run_rhs(g, u_n, vF, dt, st))) return rc;  // v = dt F(u_n)
  int* slots = o.m_carry ? state->m_slots : nullptr;
  auto slot = [&](int k) { return slots ? slots + k : nullptr; };
  int call = 0;
  // Replay records are consumed call by call; the device keeps its own count
  // per launch, so the host offsets each call by the attempts it consumes
  // (found by running the landing rule over the records).
  std::vector<int> roff(4, 0);
  if (o.replay) {
    std::vector<std::vector<double>> rhos;
    if (scheme == SWE_EPI2 || scheme == SWE_EPI3)
      rhos = {{1.0}};
    else if (scheme == SWE_EXPRB42)
      rhos = {{0.75}, {1.0}};
    else if (scheme == SWE_PEXPRB43)
      rhos = {{0.5, 1.0}, {1.0}};
    else
      rhos = {{0.5, 0.9}, {0.5, 0.9}, {1.0}};
    if ((rc = replay_split(o.replay, o.n_replay, rhos, roff))) return rc;
  }
  auto roff_at = [&](int c) { return roff[c]; };
  const double one = 1.0;
  if (scheme == SWE_EPI2 || (scheme == SWE_EPI3 && !state->have_prev)) {
    const double* v[2] = {nullptr, vF};
    double* y[1] = {B[1]};
    if ((rc = phi_call(g, u_n, dt, 1, v, 1, &one, y, o, call, slot(0), roff_at(call), st))) return rc;
    ++call;
    if ((rc = run_lincomb(g, u_np1, {{1.0, u_n}, {1.0, B[1]}}, st))) return rc;
  } else if (scheme == SWE_EXPRB42) {
    const double r1 = 0.75;
    const double* v1[2] = {nullptr, vF};
    double* y1[1] = {B[1]};
    if ((rc = phi_call(g, u_n, dt, 1, v1, 1, &r1, y1, o, call, slot(1), roff_at(call), st))) return rc;
    ++call;
    // D_2 = N(U_2) - N(u_n) = Q(U_2 - u_n); v_3 = (32/9) dt D_2
    if ((rc = run_quad(g, B[1], B[2], (32.0 / 9.0) * dt, st))) return rc;
    const double* v2[4] = {nullptr, vF, nullptr, B[2]};
    double* y2[1] = {B[3]};
    if ((rc = phi_call(g, u_n, dt, 3, v2, 1, &one, y2, o, call, slot(2), roff_at(call), st))) return rc;
    ++call;
    if ((rc = run_lincomb(g, u_np1, {{1.0, u_n}, {1.0, B[3]}}, st))) return rc;
  } else if (scheme == SWE_PEXPRB43) {
    const double r1[2] = {0.5, 1.0};
    const double* v1[2] = {nullptr, vF};
    double* y1[2] = {B[1], B[2]};
    if ((rc = phi_call(g, u_n, dt, 1, v1, 2, r1, y1, o, call, slot(1), roff_at(call), st))) return rc;
    ++call;
    if ((rc = run_quad(g, B[1], B[3], dt, st))) return rc;  // dt D_2
    if ((rc = run_quad(g, B[2], B[4], dt, st))) return rc;  // dt D_3
    if ((rc = run_lincomb(g, B[5], {{16.0, B[3]}, {-2.0, B[4]}}, st))) return rc;
    if ((rc = run_lincomb(g, B[6], {{-48.0, B[3]}, {12.0, B[4]}}, st))) return rc;
    const double* v2[5] = {nullptr, nullptr, nullptr, B[5], B[6]};
    double* y2[1] = {B[7]};
    if ((rc = phi_call(g, u_n, dt, 4, v2, 1, &one, y2, o, call, slot(2), roff_at(call), st))) return rc;
    ++call;
    // u_{n+1} = U_3 + w = u_n + Y(1) + w
    if ((rc = run_lincomb(g, u_np1, {{1.0, u_n}, {1.0, B[2]}, {1.0, B[7]}}, st))) return rc;
  } else if (scheme == SWE_EXPRB53) {
    const double r1[2] = {0.5, 0.9};
    const double* v1[2] = {nullptr, vF};
    double* y1[2] = {B[1], B[2]};
    if ((rc = phi_call(g, u_n, dt, 1, v1, 2, r1, y1, o, call, slot(1), roff_at(call), st))) return rc;
    ++call;
    if ((rc = run_quad(g, B[1], B[3], dt, st))) return rc;  // dt D_2
    const double* v2[4] = {nullptr, nullptr, nullptr, B[3]};
    double* y2[2] = {B[4], B[5]};
    if ((rc = phi_call(g, u_n, dt, 3, v2, 2, r1, y2, o, call, slot(2), roff_at(call), st))) return rc;
    ++call;
    // U_3 - u_n = Y_1(9/10) + (27/25)/(1/2)^3 Y_3(1/2) + (729/125)/(9/10)^3 Y_3(9/10)
    const double c3h = (27.0 / 25.0) / (0.5 * 0.5 * 0.5);
    const double c3n = (729.0 / 125.0) / (0.9 * 0.9 * 0.9);
    if ((rc = run_lincomb(g, B[6], {{1.0, B[2]}, {c3h, B[4]}, {c3n, B[5]}}, st))) return rc;
    if ((rc = run_quad(g, B[6], B[7], dt, st))) return rc;  // dt D_3
    if ((rc = run_lincomb(g, B[8], {{18.0, B[3]}, {-250.0 / 81.0, B[7]}}, st))) return rc;
    if ((rc = run_lincomb(g, B[9], {{-60.0, B[3]}, {500.0 / 27.0, B[7]}}, st))) return rc;
    const double* v3[5] = {nullptr, vF, nullptr, B[8], B[9]};
    double* y3[1] = {B[10]};
    if ((rc = phi_call(g, u_n, dt, 4, v3, 1, &one, y3, o, call, slot(3), roff_at(call), st))) return rc;
    ++call;
    if ((rc = run_lincomb(g, u_np1, {{1.0, u_n}, {1.0, B[10]}}, st))) return rc;
  } else {  // SWE_EPI3 with history
    // R_{n-1} = F(u_{n-1}) - F(u_n) - J_n (u_{n-1} - u_n) = Q(u_{n-1} - u_n); v_2 = (2/3) dt R
    if ((rc = run_lincomb(g, B[1], {{1.0, state->u_prev}, {-1.0, u_n}}, st))) return rc;
    if ((rc = run_quad(g, B[1], B[2], (2.0 / 3.0) * dt, st))) return rc;
    const double* v[3] = {nullptr, vF, B[2]};
    double* y[1] = {B[3]};
    if ((rc = phi_call(g, u_n, dt, 2, v, 1, &one, y, o, call, slot(1), roff_at(call), st))) return rc;
    ++call;
    if ((rc = run_lincomb(g, u_np1, {{1.0, u_n}, {1.0, B[3]}}, st))) return rc;
  }
  if (scheme == SWE_EPI3) {
    CK(cudaMemcpyAsync(state->u_prev, u_n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    state->have_prev = 1;
  }
  span.finish();
  return read_stats(g, stats, st);
}

int exprb_step_adjoint(swe_grid* g, int scheme, double dt, const double* u_n, const phi_attempt* trace,
                       int n_trace, const double* lam_np1, double* lam_n, const phi_opts* opts,
                       phi_stats* stats, void* stream) {
  if (!g || !u_n || !trace || !lam_np1 || !lam_n)
    return fail(SWE_ERR_INVALID_ARG, "exprb_step_adjoint: NULL argument");
  if (lam_n == lam_np1 || lam_n == u_n) return fail(SWE_ERR_INVALID_ARG, "exprb_step_adjoint: lam_n must not alias");
  if (scheme != SWE_EPI2 && scheme != SWE_EXPRB42 && scheme != SWE_PEXPRB43 && scheme != SWE_EXPRB53)
    return fail(SWE_ERR_INVALID_ARG, "exprb_step_adjoint: EPI2, exprb42, pexprb43 and exprb53 are supported");
  if (n_trace < 1) return fail(SWE_ERR_INVALID_ARG, "exprb_step_adjoint: empty trace");
  int rc;
  phi_opts o;
  if ((rc = resolve_opts(opts, o))) return rc;
  if (o.precision != 0) return fail(SWE_ERR_INVALID_ARG, "exprb_step_adjoint: FP64 only (precision = 0)");
  if (o.iom != 2) return fail(SWE_ERR_INVALID_ARG, "exprb_step_adjoint: IOM2 only (iom = 2)");
  if ((rc = ensure_workspace(g))) return rc;
  if ((rc = ensure_adjoint(g))) return rc;
  cudaStream_t st = S(stream);
  // the scheme's phi calls: p of each call
  int ncalls = 1;
  int pc[3] = {1, 0, 0};
  if (scheme == SWE_EXPRB42) {
    ncalls = 2;
    pc[1] = 3;
  } else if (scheme == SWE_PEXPRB43) {
    ncalls = 2;
    pc[1] = 4;
  } else if (scheme == SWE_EXPRB53) {
    ncalls = 3;
    pc[1] = 3;
    pc[2] = 4;
  }
  TapePlan P;
  if ((rc = plan_tape(trace, n_trace, ncalls, P))) return rc;
  TapeCall tapes[3];
  if ((rc = alloc_tapes(g, P, pc, ncalls, tapes, st))) return rc;
  // forward replay with tapes: the same calls as exprb_step
  o.replay = P.replay.data();
  o.n_replay = (int)(P.replay.size() / 3);
  if ((rc = stage_replay(g, o, st))) return rc;
  const size_t n = (size_t)4 * g->T.ng;
  double* B[ADJ_VECS];
  for (int k = 0; k < ADJ_VECS; ++k) B[k] = g->avec + (size_t)k * n;
  double* vF = B[0];  // dt F(u_n)
  double* yw = B[1];  // forward output of the last call (not needed)
  ProfSpan span(g, st, &g->call_ev);
  CK(cudaMemsetAsync(g->stats, 0, sizeof(DevStats), st));
  CK(cudaMemsetAsync(g->adj_status, 0, sizeof(int), st));
  if ((rc = prepare_lin(g, u_n, o, st))) return rc;
  if ((rc = run_rhs(g, u_n, vF, dt, st))) return rc;
  const double one = 1.0;
  auto call = [&](int c, int p, const double* const* v, int ns, const double* rho, double* const* y) {
    return phi_call(g, u_n, dt, p, v, ns, rho, y, o, c, nullptr, P.first[c], st, &tapes[c]);
  };
  // exprb53 stage weights of U_3 (Eq. eq3.13 with the rho^3 of Y_3)
  const double c3h = (27.0 / 25.0) / (0.5 * 0.5 * 0.5);
  const double c3n = (729.0 / 125.0) / (0.9 * 0.9 * 0.9);
  if (scheme == SWE_EPI2) {
    const double* v[2] = {nullptr, vF};
    double* y[1] = {yw};
    if ((rc = call(0, 1, v, 1, &one, y))) return rc;
  } else if (scheme == SWE_EXPRB42) {
    const double r1 = 0.75;
    const double* v1[2] = {nullptr, vF};
    double* y1[1] = {B[2]};                                          // Y1
    if ((rc = call(0, 1, v1, 1, &r1, y1))) return rc;
    if ((rc = run_quad(g, B[2], B[3], (32.0 / 9.0) * dt, st))) return rc;  // v_3
    const double* v2[4] = {nullptr, vF, nullptr, B[3]};
    double* y2[1] = {yw};
    if ((rc = call(1, 3, v2, 1, &one, y2))) return rc;
  } else if (scheme == SWE_PEXPRB43) {
    const double r1[2] = {0.5, 1.0};
    const double* v1[2] = {nullptr, vF};
    double* y1[2] = {B[2], B[3]};                                    // Y(1/2), Y(1)
    if ((rc = call(0, 1, v1, 2, r1, y1))) return rc;
    if ((rc = run_quad(g, B[2], B[4], dt, st))) return rc;           // dt D_2
    if ((rc = run_quad(g, B[3], B[5], dt, st))) return rc;           // dt D_3
    if ((rc = run_lincomb(g, B[6], {{16.0, B[4]}, {-2.0, B[5]}}, st))) return rc;
    if ((rc = run_lincomb(g, B[7], {{-48.0, B[4]}, {12.0, B[5]}}, st))) return rc;
    const double* v2[5] = {nullptr, nullptr, nullptr, B[6], B[7]};
    double* y2[1] = {yw};
    if ((rc = call(1, 4, v2, 1, &one, y2))) return rc;
  } else {  // SWE_EXPRB53
    const double r1[2] = {0.5, 0.9};
    const double* v1[2] = {nullptr, vF};
    double* y1[2] = {B[2], B[3]};                                    // Y_1(1/2), Y_1(9/10)
    if ((rc = call(0, 1, v1, 2, r1, y1))) return rc;
    if ((rc = run_quad(g, B[2], B[4], dt, st))) return rc;           // dt D_2
    const double* v2[4] = {nullptr, nullptr, nullptr, B[4]};
    double* y2[2] = {B[5], B[6]};                                    // Y_3(1/2), Y_3(9/10)
    if ((rc = call(1, 3, v2, 2, r1, y2))) return rc;
    if ((rc = run_lincomb(g, B[7], {{1.0, B[3]}, {c3h, B[5]}, {c3n, B[6]}}, st))) return rc;  // U_3 - u_n
    if ((rc = run_quad(g, B[7], B[8], dt, st))) return rc;           // dt D_3
    if ((rc = run_lincomb(g, B[9], {{18.0, B[4]}, {-250.0 / 81.0, B[8]}}, st))) return rc;
    if ((rc = run_lincomb(g, B[10], {{-60.0, B[4]}, {500.0 / 27.0, B[8]}}, st))) return rc;
    const double* v3[5] = {nullptr, vF, nullptr, B[9], B[10]};
    double* y3[1] = {yw};
    if ((rc = call(2, 4, v3, 1, &one, y3))) return rc;
  }
  // reverse (the tape's scalars are checked by the reverse launch against the
  // layout, so a failed recomputation cannot send it out of bounds; its
  // status is read once at the end).  Adjoint vectors: VB1 of v_1 = dt F(u_n); the rest per scheme.
  double* VB1 = B[11];
  double* T1 = B[12];
  double* T2 = B[13];
  double* T3 = B[14];
  double* T4 = B[15];
  double* auxq = B[1];  // aux planes for Q'^T (yw is not needed any more)
  CK(cudaMemcpyAsync(lam_n, lam_np1, n * sizeof(double), cudaMemcpyDeviceToDevice, st));  // u_{n+1} = u_n + ...
  CK(cudaMemsetAsync(VB1, 0, n * sizeof(double), st));
  auto zero = [&](double* x) { return cudaMemsetAsync(x, 0, n * sizeof(double), st); };
  if (scheme == SWE_EPI2) {
    const double* yb[1] = {lam_np1};
    double* vb[2] = {nullptr, VB1};
    if ((rc = adj_call(g, tapes[0], u_n, dt, yb, 1, vb, lam_n, st))) return rc;
  } else if (scheme == SWE_EXPRB42) {
    CK(zero(T1));
    {
      const double* yb[1] = {lam_np1};
      double* vb[4] = {nullptr, VB1, nullptr, T1};                   // T1: adjoint of v_3
      if ((rc = adj_call(g, tapes[1], u_n, dt, yb, 1, vb, lam_n, st))) return rc;
    }
    // v_3 = (32/9) dt Q(Y1): adjoint of Y1 into T2
    if ((rc = run_transposed<MODE_QT>(g, B[2], T1, (32.0 / 9.0) * dt, 0, T2, auxq, st))) return rc;
    {
      const double* yb[1] = {T2};
      double* vb[2] = {nullptr, VB1};
      if ((rc = adj_call(g, tapes[0], u_n, dt, yb, 1, vb, lam_n, st))) return rc;
    }
  } else if (scheme == SWE_PEXPRB43) {
    CK(zero(T1));
    CK(zero(T2));
    {
      const double* yb[1] = {lam_np1};
      double* vb[5] = {nullptr, nullptr, nullptr, T1, T2};           // adjoints of v_3, v_4
      if ((rc = adj_call(g, tapes[1], u_n, dt, yb, 1, vb, lam_n, st))) return rc;
    }
    // v_3 = 16 dD_2 - 2 dD_3, v_4 = -48 dD_2 + 12 dD_3 (dD = dt D):
    // adjoints of dt D_2 (T3) and dt D_3 (T4)
    if ((rc = run_lincomb(g, T3, {{16.0, T1}, {-48.0, T2}}, st))) return rc;
    if ((rc = run_lincomb(g, T4, {{-2.0, T1}, {12.0, T2}}, st))) return rc;
    // dt D_2 = dt Q(Y(1/2)), dt D_3 = dt Q(Y(1)); u_{n+1} = u_n + Y(1) + w
    if ((rc = run_transposed<MODE_QT>(g, B[2], T3, dt, 0, T1, auxq, st))) return rc;       // Ybar(1/2)
    CK(cudaMemcpyAsync(T2, lam_np1, n * sizeof(double), cudaMemcpyDeviceToDevice, st));   // Ybar(1)
    if ((rc = run_transposed<MODE_QT>(g, B[3], T4, dt, 1, T2, auxq, st))) return rc;
    {
      const double* yb[2] = {T1, T2};
      double* vb[2] = {nullptr, VB1};
      if ((rc = adj_call(g, tapes[0], u_n, dt, yb, 2, vb, lam_n, st))) return rc;
    }
  } else {  // SWE_EXPRB53
    CK(zero(T1));
    CK(zero(T2));
    {
      const double* yb[1] = {lam_np1};
      double* vb[5] = {nullptr, VB1, nullptr, T1, T2};               // adjoints of v_1, v_3, v_4
      if ((rc = adj_call(g, tapes[2], u_n, dt, yb, 1, vb, lam_n, st))) return rc;
    }
    // v_3 = 18 dD_2 - 250/81 dD_3, v_4 = -60 dD_2 + 500/27 dD_3
    if ((rc = run_lincomb(g, T3, {{18.0, T1}, {-60.0, T2}}, st))) return rc;                // of dt D_2
    if ((rc = run_lincomb(g, T4, {{-250.0 / 81.0, T1}, {500.0 / 27.0, T2}}, st))) return rc;  // of dt D_3
    // dt D_3 = dt Q(U_3 - u_n), U_3 - u_n = Y_1(9/10) + c3h Y_3(1/2) + c3n Y_3(9/10)
    if ((rc = run_transposed<MODE_QT>(g, B[7], T4, dt, 0, T1, auxq, st))) return rc;       // of U_3 - u_n
    if ((rc = run_lincomb(g, T2, {{c3h, T1}}, st))) return rc;                              // of Y_3(1/2)
    if ((rc = run_lincomb(g, T4, {{c3n, T1}}, st))) return rc;                              // of Y_3(9/10)
    {
      const double* yb[2] = {T2, T4};
      double* vb[4] = {nullptr, nullptr, nullptr, T3};               // += adjoint of dt D_2
      if ((rc = adj_call(g, tapes[1], u_n, dt, yb, 2, vb, lam_n, st))) return rc;
    }
    // dt D_2 = dt Q(Y_1(1/2)); Y_1(9/10) has the adjoint of U_3 - u_n (T1)
    if ((rc = run_transposed<MODE_QT>(g, B[2], T3, dt, 0, T2, auxq, st))) return rc;       // of Y_1(1/2)
    {
      const double* yb[2] = {T2, T1};
      double* vb[2] = {nullptr, VB1};
      if ((rc = adj_call(g, tapes[0], u_n, dt, yb, 2, vb, lam_n, st))) return rc;
    }
  }
  // v_1 = dt F(u_n): lam_n += dt J(u_n)^T VB1
  if ((rc = run_transposed<MODE_JT>(g, u_n, VB1, dt, 1, lam_n, nullptr, st))) return rc;
  span.finish();
  DevStats ds;
  int ast = SWE_OK;
  CK(cudaMemcpyAsync(&ds, g->stats, sizeof(DevStats), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ast, g->adj_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (stats) {
    stats->n_jv = ds.n_jv;
    stats->n_substeps = ds.n_sub;
    stats->n_reject = ds.n_rej;
    stats->m_last = ds.m_last;
    stats->m_max_used = ds.m_max_used;
    stats->status = ds.status != SWE_OK ? ds.status : ast;
    stats->n_trace = 0;
  }
  if (ds.status != SWE_OK) return fail(ds.status, "exprb_step_adjoint: the forward recomputation failed");
  if (ast != SWE_OK) return fail(ast, "exprb_step_adjoint: the reverse launch reported an error");
  return SWE_OK;
}

// ---------------------------------------------------------------------------
// ensembles
// ---------------------------------------------------------------------------
static int ens_upload_split(swe_ensemble* E) {
  int b = 0;
  std::vector<int> blk(E->nb_alloc, -1);
  E->nb.assign(E->nmem, 0);
  for (size_t g = 0; g < E->groups.size(); ++g) {
    const std::vector<int>& mem = E->groups[g];
    const int nbg = E->gnb[g];
    if (mem.empty() || nbg < 1) return fail(SWE_ERR_INVALID_ARG, "ensemble: empty group");
    if (b + nbg > E->nblocks) return fail(SWE_ERR_INVALID_ARG, "ensemble block split exceeds the launch");
    for (size_t k = 0; k < mem.size(); ++k) {
      EnsMember& M = E->hmem[mem[k]];
      M.b0 = b;
      M.nb = nbg;
      M.next = k + 1 < mem.size() ? mem[k + 1] : -1;
      E->nb[mem[k]] = nbg;
    }
    for (int k = 0; k < nbg; ++k) blk[b + k] = mem[0];
    b += nbg;
  }
  E->nblocks = b;
  CK(cudaMemcpy(E->dblk, blk.data(), (size_t)b * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(E->dmem, E->hmem.data(), E->hmem.size() * sizeof(EnsMember), cudaMemcpyHostToDevice));
  return SWE_OK;
}

// Blocks proportional to weights, at least one each, summing to total
// (largest remainders).
static std::vector<int> ens_split(const std::vector<double>& w, int total) {
  const int n = (int)w.size();
  double sum = 0.0;
  for (double x : w) sum += x;
  std::vector<int> nb(n, 1);
  int left = total - n;
  std::vector<std::pair<double, int>> rem;
  int used = 0;
  for (int m = 0; m < n; ++m) {
    double share = sum > 0 ? left * w[m] / sum : 0.0;
    int k = (int)share;
    nb[m] += k;
    used += k;
    rem.push_back({share - k, m});
  }
  std::sort(rem.begin(), rem.end(), [](auto& a, auto& b) { return a.first > b.first; });
  for (int r = 0; r < left - used && r < n; ++r) nb[rem[r].second] += 1;
  return nb;
}

// Split minimising the predicted longest group time, with member m taking
// t_m(b) = s[m] + p[m] / b on b blocks: bisection on the target time T, each
// member getting the fewest blocks that meet T; blocks left over go, one at a
// time, to the member predicted slowest.
static std::vector<int> ens_split_model(const std::vector<double>& s, const std::vector<double>& p, int total) {
  const int n = (int)s.size();
  auto need = [&](double T, std::vector<int>& nb) {
    long long sum = 0;
    for (int m = 0; m < n; ++m) {
      const double room = T - s[m];
      long long b = room > 0.0 ? (long long)std::ceil(p[m] / room) : (long long)total + 1;
      b = std::max(1LL, b);
      nb[m] = (int)std::min<long long>(b, total);
      sum += b;
    }
    return sum;
  };
  std::vector<int> nb(n, 1);
  double lo = 0.0, hi = 0.0;
  for (int m = 0; m < n; ++m) hi = std::max(hi, s[m] + p[m]);  // everyone on one block
  for (int it = 0; it < 100; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (need(mid, nb) <= total)
      hi = mid;
    else
      lo = mid;
  }
  need(hi, nb);
  int used = std::accumulate(nb.begin(), nb.end(), 0);
  while (used < total) {
    int worst = 0;
    double tw = -1.0;
    for (int m = 0; m < n; ++m) {
      const double t = s[m] + p[m] / nb[m];
      if (t > tw) {
        tw = t;
        worst = m;
      }
    }
    ++nb[worst];
    ++used;
  }
  return nb;
}

extern "C" int swe_ensemble_create(swe_grid* const* grids, int nmem, const double* dt, const int* nsteps,
                                   const phi_opts* opts, swe_ensemble** out) {
  if (!grids || !dt || !nsteps || !out || nmem < 1) return fail(SWE_ERR_INVALID_ARG, "ensemble: bad arguments");
  *out = nullptr;
  phi_opts o;
  int rc = resolve_opts(opts, o);
  if (rc) return rc;
  if (o.precision != 0 || o.replay || o.iom != 2)
    return fail(SWE_ERR_INVALID_ARG, "ensemble: FP64, IOM2, without replay only");
  int NB = 0, threads = 0, nb_alloc = 0;
  if (ens_max_blocks(0, &NB, &threads, nullptr) != 0) return fail(SWE_ERR_CUDA, "ensemble: occupancy query failed");
  if (nmem > NB) return fail(SWE_ERR_INVALID_ARG, "ensemble: more members than co-resident blocks");
  for (int sh = 0; sh < ENS_SHAPES; ++sh) {
    int nbs = 0, ts = 0;
    if (ens_max_blocks(sh, &nbs, &ts, nullptr) == 0) nb_alloc = std::max(nb_alloc, nbs);
  }
  for (int m = 0; m < nmem; ++m) {
    if (!grids[m] || !grids[m]->dtab || !(dt[m] > 0.0) || nsteps[m] < 0)
      return fail(SWE_ERR_INVALID_ARG, "ensemble: each member needs a device grid, dt > 0, nsteps >= 0");
  }
  std::unique_ptr<swe_ensemble> E(new swe_ensemble());
  E->nmem = nmem;
  E->shape = 0;
  E->nblocks = NB;
  E->nb_alloc = nb_alloc;
  E->grids.assign(grids, grids + nmem);
  // workspace layout per member (doubles): Vbuf (KMAX+1)n, W (PMAX+1)n, tmp 8ng, Lring 3n,
  // Zbuf n, aux 4ng, part NB*NRED, u n, vF n, v3 n, y1 n, w n, tmpS 8ng  + ctrl, slots
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  std::vector<size_t> off(nmem);
  size_t total = 0;
  for (int m = 0; m < nmem; ++m) {
    const size_t ng = grids[m]->T.ng, n = 4 * ng;
    off[m] = total;
    size_t d = (size_t)(KMAX + 1) * n + (size_t)(PMAX + 1) * n + 8 * ng + 3 * n + n + 4 * ng +
               (size_t)nb_alloc * NRED + 5 * n + 8 * ng;
    total += al(d * 8) + al(sizeof(PhiCtrl));
  }
  size_t nstates = 0;
  for (int m = 0; m < nmem; ++m) {
    E->state_off.push_back(nstates);
    nstates += (size_t)4 * grids[m]->T.ng;
  }
  cudaError_t e = cudaMalloc(&E->dws, total);
  if (e == cudaSuccess) e = cudaMalloc(&E->dmem, (size_t)nmem * sizeof(EnsMember));
  if (e == cudaSuccess) e = cudaMalloc(&E->dblk, (size_t)nb_alloc * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&E->dsync, (size_t)nmem * sizeof(GridSync));
  if (e == cudaSuccess) e = cudaMalloc(&E->dstats, (size_t)nmem * sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMalloc(&E->backup, nstates * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&E->dslots, (size_t)2 * nmem * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&E->dslots_backup, (size_t)2 * nmem * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(E->dslots, 0, (size_t)2 * nmem * sizeof(int));
  if (e != cudaSuccess) {
    swe_ensemble_destroy(E.release());
    return fail(SWE_ERR_NOMEM, std::string("ensemble allocation failed: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemset(E->dws, 0, total)) != cudaSuccess) {
    swe_ensemble_destroy(E.release());
    return cuda_fail(e, "cudaMemset(ensemble)");
  }
  E->hmem.resize(nmem);
  std::vector<double> weight(nmem);
  for (int m = 0; m < nmem; ++m) {
    swe_grid* g = grids[m];
    const size_t ng = g->T.ng, n = 4 * ng;
    double* p = (double*)((char*)E->dws + off[m]);
    auto take = [&](size_t cnt) {
      double* q = p;
      p += cnt;
      return q;
    };
    EnsMember& M = E->hmem[m];
    std::memset(&M, 0, sizeof(M));
    double* Vbuf = take((size_t)(KMAX + 1) * n);
    double* W = take((size_t)(PMAX + 1) * n);
    double* tmp = take(8 * ng);
    double* Lring = take(3 * n);
    double* Zbuf = take(n);
    double* aux = take(4 * ng);
    double* part = take((size_t)nb_alloc * NRED);
    M.u = take(n);
    M.vF = take(n);
    M.v3 = take(n);
    M.y1 = take(n);
    M.w = take(n);
    M.tmpS = take(8 * ng);
    M.aux = aux;
    char* q = (char*)E->dws + off[m] + al(((size_t)(KMAX + 1) * n + (size_t)(PMAX + 1) * n + 8 * ng + 3 * n +
                                             n + 4 * ng + (size_t)nb_alloc * NRED + 5 * n + 8 * ng) * 8);
    PhiCtrl* ctrl = (PhiCtrl*)q;
    int* slots = E->dslots + 2 * m;
    M.dt = dt[m];
    M.nsteps = nsteps[m];
    for (int c = 0; c < 2; ++c) {
      PhiArgs& a = c == 0 ? M.c1 : M.c2;
      a.T = g->T;
      a.u_lin = M.u;
      a.aux = aux;
      a.dt = dt[m];
      a.ns = 1;
      a.Vbuf = Vbuf;
      a.W = W;
      a.tmp = tmp;
      a.Lring = Lring;
      a.Zbuf = Zbuf;
      a.part = part;
      a.ctrl = ctrl;
      a.sync = E->dsync + m;
      a.stats = E->dstats + m;
      a.prof = nullptr;
      a.trace = nullptr;
      a.trace_cap = 0;
      a.call_index = c;
      a.m_slot = o.m_carry ? slots + c : nullptr;
      a.replay = nullptr;
      a.n_replay = 0;
      a.tol = o.tol;
      a.delta = o.delta;
      a.gamma = o.gamma;
      a.kappa = o.kappa;
      a.tol_mode = o.tol_mode;
      a.m_init = o.m_init;
      a.m_max = o.m_max;
      a.max_reject = o.max_reject;
      a.max_substeps = o.max_substeps;
      a.iom = 2;
      a.nA = g->host.nA;
    }
    M.c1.p = 1;
    M.c1.rho[0] = 0.75;
    M.c1.v[1] = M.vF;
    M.c1.y_out[0] = M.y1;
    M.c2.p = 3;
    M.c2.rho[0] = 1.0;
    M.c2.v[1] = M.vF;
    M.c2.v[3] = M.v3;
    M.c2.y_out[0] = M.w;
    // work model: total Krylov iterations grow with dt * 2^level per step,
    // i.e. with 2^level * (simulated time); cost per iteration with cells
    weight[m] = (double)ng * std::pow(2.0, g->host.level) * dt[m] * (nsteps[m] > 0 ? nsteps[m] : 0) + 1.0;
  }
  E->weight = weight;
  E->groups.clear();
  for (int m = 0; m < nmem; ++m) E->groups.push_back({m});
  E->gnb = ens_split(weight, NB);
  if ((rc = ens_upload_split(E.get()))) {
    swe_ensemble_destroy(E.release());
    return rc;
  }
  *out = E.release();
  return SWE_OK;
}

extern "C" void swe_ensemble_destroy(swe_ensemble* E) {
  if (!E) return;
  if (E->dws) cudaFree(E->dws);
  if (E->dmem) cudaFree(E->dmem);
  if (E->dblk) cudaFree(E->dblk);
  if (E->dsync) cudaFree(E->dsync);
  if (E->dstats) cudaFree(E->dstats);
  if (E->backup) cudaFree(E->backup);
  if (E->dslots) cudaFree(E->dslots);
  if (E->dslots_backup) cudaFree(E->dslots_backup);
  delete E;
}

extern "C" int swe_ensemble_set_state(swe_ensemble* E, int m, const double* u, void* stream) {
  if (!E || m < 0 || m >= E->nmem || !u) return fail(SWE_ERR_INVALID_ARG, "ensemble_set_state: bad arguments");
  CK(cudaMemcpyAsync(E->hmem[m].u, u, (size_t)4 * E->grids[m]->T.ng * sizeof(double),
                     cudaMemcpyDeviceToDevice, S(stream)));
  return SWE_OK;
}

extern "C" int swe_ensemble_get_state(swe_ensemble* E, int m, double* u, void* stream) {
  if (!E || m < 0 || m >= E->nmem || !u) return fail(SWE_ERR_INVALID_ARG, "ensemble_get_state: bad arguments");
  CK(cudaMemcpyAsync(u, E->hmem[m].u, (size_t)4 * E->grids[m]->T.ng * sizeof(double),
                     cudaMemcpyDeviceToDevice, S(stream)));
  return SWE_OK;
}

extern "C" int swe_ensemble_reset(swe_ensemble* E, void* stream) {
  if (!E) return fail(SWE_ERR_INVALID_ARG, "ensemble is NULL");
  CK(cudaMemsetAsync(E->dslots, 0, (size_t)2 * E->nmem * sizeof(int), S(stream)));
  return SWE_OK;
}

extern "C" int swe_ensemble_run(swe_ensemble* E, void* stream) {
  if (!E) return fail(SWE_ERR_INVALID_ARG, "ensemble is NULL");
  cudaStream_t st = S(stream);
  CK(cudaMemsetAsync(E->dsync, 0, (size_t)E->nmem * sizeof(GridSync), st));
  CK(cudaMemsetAsync(E->dstats, 0, (size_t)E->nmem * sizeof(DevStats), st));
  int e = launch_ens_kernel(E->shape, E->dmem, E->dblk, E->nblocks, st);
  if (e != 0) return cuda_fail((cudaError_t)e, "cudaLaunchKernelEx(ens_kernel)");
  return SWE_OK;
}

extern "C" int swe_ensemble_stats(swe_ensemble* E, phi_stats* stats, double* member_ms, int* member_blocks,
                                  void* stream) {
  if (!E) return fail(SWE_ERR_INVALID_ARG, "ensemble is NULL");
  CK(cudaStreamSynchronize(S(stream)));
  std::vector<DevStats> ds(E->nmem);
  std::vector<EnsMember> hm(E->nmem);
  CK(cudaMemcpy(ds.data(), E->dstats, ds.size() * sizeof(DevStats), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hm.data(), E->dmem, hm.size() * sizeof(EnsMember), cudaMemcpyDeviceToHost));
  for (int m = 0; m < E->nmem; ++m) {
    if (stats) {
      stats[m].n_jv = ds[m].n_jv;
      stats[m].n_substeps = ds[m].n_sub;
      stats[m].n_reject = ds[m].n_rej;
      stats[m].m_last = ds[m].m_last;
      stats[m].m_max_used = ds[m].m_max_used;
      stats[m].status = ds[m].status;
      stats[m].n_trace = 0;
    }
    if (member_ms) member_ms[m] = 1e-6 * (double)(hm[m].t1 - hm[m].t0);
    if (member_blocks) member_blocks[m] = E->nb[m];
  }
  return SWE_OK;
}

// Groups and blocks for `total` blocks from per-member fits t_m(b) = s_m +
// p_m / b [ms] (members of a group run one after the other on its blocks, so
// a group takes sum s + (sum p) / b).  Starting from one member per group and
// the split that minimises the predicted longest group (time T), members that
// would take at most T/2 on one block are stacked, longest first, into the
// first group whose one-block time stays within T; the freed blocks are
// split again.  Repeated while the predicted longest group gets shorter.
static void ens_plan(const std::vector<double>& s, const std::vector<double>& p, int total,
                     std::vector<std::vector<int>>& groups, std::vector<int>& gnb) {
  const int n = (int)s.size();
  auto split = [&](const std::vector<std::vector<int>>& gr, std::vector<int>& nb) {
    std::vector<double> sg(gr.size(), 0.0), pg(gr.size(), 0.0);
    for (size_t g = 0; g < gr.size(); ++g)
      for (int m : gr[g]) {
        sg[g] += s[m];
        pg[g] += p[m];
      }
    nb = ens_split_model(sg, pg, total);
    double T = 0.0;
    for (size_t g = 0; g < gr.size(); ++g) T = std::max(T, sg[g] + pg[g] / nb[g]);
    return T;
  };
  groups.clear();
  for (int m = 0; m < n; ++m) groups.push_back({m});
  double T = split(groups, gnb);
  for (int pass = 0; pass < 4; ++pass) {
    std::vector<int> small, big;
    for (int m = 0; m < n; ++m) (s[m] + p[m] <= 0.5 * T ? small : big).push_back(m);
    std::sort(small.begin(), small.end(), [&](int a, int b) { return s[a] + p[a] > s[b] + p[b]; });
    std::vector<std::vector<int>> bins;
    std::vector<double> load;
    for (int m : small) {
      const double t1 = s[m] + p[m];
      size_t k = 0;
      while (k < bins.size() && load[k] + t1 > T) ++k;
      if (k == bins.size()) {
        bins.push_back({});
        load.push_back(0.0);
      }
      bins[k].push_back(m);
      load[k] += t1;
    }
    std::vector<std::vector<int>> cand = bins;
    for (int m : big) cand.push_back({m});
    if ((int)cand.size() > total || cand.size() == groups.size()) break;
    std::vector<int> nb;
    const double Tn = split(cand, nb);
    if (!(Tn < T)) break;
    groups = cand;
    gnb = nb;
    T = Tn;
  }
}

extern "C" int swe_ensemble_tune(swe_ensemble* E, int rounds, void* stream) {
  if (!E || rounds < 0) return fail(SWE_ERR_INVALID_ARG, "ensemble_tune: bad arguments");
  if (rounds == 0) return SWE_OK;
  cudaStream_t st = S(stream);
  for (int m = 0; m < E->nmem; ++m)
    CK(cudaMemcpyAsync(E->backup + E->state_off[m], E->hmem[m].u, (size_t)4 * E->grids[m]->T.ng * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(E->dslots_backup, E->dslots, (size_t)2 * E->nmem * sizeof(int), cudaMemcpyDeviceToDevice, st));
  const int nm = E->nmem;
  int best_shape = E->shape;
  std::vector<std::vector<int>> best_groups = E->groups;
  std::vector<int> best_gnb = E->gnb;
  double best_t = -1.0;
  // fits t = s + p / b per member; p is carried between shapes in thread-blocks
  // (p x threads), s as it is
  std::vector<double> fs(nm, 0.0), fpt(nm, 0.0);
  bool have_fit = false;
  for (int sh = 0; sh < ENS_SHAPES; ++sh) {
    int NB = 0, threads = 0;
    if (ens_max_blocks(sh, &NB, &threads, nullptr) != 0 || NB < 1) continue;
    E->shape = sh;
    E->nblocks = NB;
    std::vector<double> sv(nm), pv(nm);
    if (have_fit) {
      for (int m = 0; m < nm; ++m) {
        sv[m] = fs[m];
        pv[m] = fpt[m] / threads;
      }
      ens_plan(sv, pv, NB, E->groups, E->gnb);
    } else {
      E->groups.clear();
      for (int m = 0; m < nm; ++m) E->groups.push_back({m});
      if (NB < nm) continue;
      E->gnb = ens_split(E->weight, NB);
    }
    if ((int)E->groups.size() > NB) continue;
    // per member: the last two (blocks, ms) measurements of this shape
    std::vector<std::pair<int, double>> last1(nm, {0, 0.0}), last2(nm, {0, 0.0});
    for (int r = 0; r < rounds; ++r) {
      E->nblocks = NB;
      int rc = ens_upload_split(E);
      if (rc) return rc;
      if ((rc = swe_ensemble_run(E, stream))) return rc;
      std::vector<phi_stats> ps(nm);
      std::vector<double> ms(nm);
      if ((rc = swe_ensemble_stats(E, ps.data(), ms.data(), nullptr, stream))) return rc;
      for (int m = 0; m < nm; ++m)
        if (ps[m].status != SWE_OK) return fail(ps[m].status, "ensemble_tune: a member failed");
      std::vector<EnsMember> hm(nm);
      CK(cudaMemcpy(hm.data(), E->dmem, hm.size() * sizeof(EnsMember), cudaMemcpyDeviceToHost));
      double tmax = 0.0;
      for (const auto& g : E->groups)
        tmax = std::max(tmax, 1e-6 * (double)(hm[g.back()].t1 - hm[g.front()].t0));
      if (best_t < 0.0 || tmax < best_t) {
        best_t = tmax;
        best_shape = sh;
        best_groups = E->groups;
        best_gnb = E->gnb;
      }
      for (int m = 0; m < nm; ++m) {
        last2[m] = last1[m];
        last1[m] = {E->nb[m], ms[m]};
        double sm = 0.0, pm = ms[m] * E->nb[m];  // one measurement: all parallel
        const int b1 = last1[m].first, b2 = last2[m].first;
        if (b2 > 0 && b2 != b1) {
          const double t1 = last1[m].second, t2 = last2[m].second;
          const double x1 = 1.0 / b1, x2 = 1.0 / b2;
          const double pf = (t1 - t2) / (x1 - x2);
          const double sf = t1 - pf * x1;
          if (pf > 0.0 && sf >= 0.0) {
            sm = sf;
            pm = pf;
          }
        }
        sv[m] = sm;
        pv[m] = pm;
        fs[m] = sm;
        fpt[m] = pm * threads;
      }
      have_fit = true;
      for (int m = 0; m < nm; ++m)
        CK(cudaMemcpyAsync(E->hmem[m].u, E->backup + E->state_off[m],
                           (size_t)4 * E->grids[m]->T.ng * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(E->dslots, E->dslots_backup, (size_t)2 * nm * sizeof(int), cudaMemcpyDeviceToDevice, st));
      CK(cudaStreamSynchronize(st));
      ens_plan(sv, pv, NB, E->groups, E->gnb);
    }
  }
  // keep the best measured launch (shape, groups, split)
  E->shape = best_shape;
  E->groups = best_groups;
  E->gnb = best_gnb;
  int NB = 0, threads = 0;
  if (ens_max_blocks(best_shape, &NB, &threads, nullptr) != 0) return fail(SWE_ERR_CUDA, "ensemble: occupancy query failed");
  E->nblocks = NB;
  return ens_upload_split(E);
}

extern "C" int swe_ensemble_shape(const swe_ensemble* E, int* threads, int* blocks_per_sm, int* nblocks,
                                  int* ngroups, int* member_group) {
  if (!E) return fail(SWE_ERR_INVALID_ARG, "ensemble is NULL");
  int NB = 0, t = 0, per = 0;
  if (ens_max_blocks(E->shape, &NB, &t, &per) != 0) return fail(SWE_ERR_CUDA, "ensemble: occupancy query failed");
  if (threads) *threads = t;
  if (blocks_per_sm) *blocks_per_sm = per;
  if (nblocks) *nblocks = E->nblocks;
  if (ngroups) *ngroups = (int)E->groups.size();
  if (member_group)
    for (size_t g = 0; g < E->groups.size(); ++g)
      for (int m : E->groups[g]) member_group[m] = (int)g;
  return SWE_OK;
}

extern "C" int swe_ensemble_work(swe_ensemble* E, double* flop, void* stream) {
  if (!E || !flop) return fail(SWE_ERR_INVALID_ARG, "ensemble and flop are required");
  CK(cudaStreamSynchronize(S(stream)));
  std::vector<DevStats> ds(E->nmem);
  CK(cudaMemcpy(ds.data(), E->dstats, ds.size() * sizeof(DevStats), cudaMemcpyDeviceToHost));
  double f = 0.0;
  for (int m = 0; m < E->nmem; ++m)
    f += (double)E->grids[m]->T.ng *
         (kFlopIter * (double)ds[m].n_iter + kFlopWjv * (double)ds[m].n_wjv + kFlopComb * (double)ds[m].comb_terms);
  *flop = f;
  return SWE_OK;
}

int swe_profile_enable(swe_grid* g, int on) {
  if (!g) return fail(SWE_ERR_INVALID_ARG, "grid is NULL");
  int rc = ensure_workspace(g);
  if (rc) return rc;
  if (on) {
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(g->dprof, 0, sizeof(DevProfile)));
    g->phi_ev.clear();
    g->call_ev.clear();
    g->ev_used = 0;
    g->kernel_launches = 0;
  }
  g->prof_on = on != 0;
  return SWE_OK;
}

int swe_profile_read(swe_grid* g, swe_profile* out, void* stream) {
  if (!g || !out) return fail(SWE_ERR_INVALID_ARG, "grid and out are required");
  std::memset(out, 0, sizeof(*out));
  if (!g->dprof) return SWE_OK;
  CK(cudaStreamSynchronize(S(stream)));
  CK(cudaDeviceSynchronize());
  DevProfile dp;
  CK(cudaMemcpy(&dp, g->dprof, sizeof(DevProfile), cudaMemcpyDeviceToHost));
  for (auto& pr : g->phi_ev) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
    out->phi_ms += ms;
  }
  for (auto& pr : g->call_ev) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
    out->call_ms += ms;
  }
  out->phi_launches = dp.launches;
  out->kernel_launches = g->kernel_launches;
  out->iom2_iterations = dp.iters;
  out->w_jv = dp.wjv;
  out->comb_terms = dp.comb_terms;
  out->phi_flop = dp.flop;
  out->phi_bytes = dp.bytes;
  out->phi_table_bytes = dp.table_bytes;
  for (int k = 0; k < 10; ++k) out->phase_ms[k] = 1e-6 * (double)dp.phase_ns[k];
  return SWE_OK;
}

int swe_selftest_wait(int64_t limit_ns, int preset_abort, int* status_out, void* stream) {
  if (!status_out || limit_ns < 1000 || limit_ns > 1000000000) return fail(SWE_ERR_INVALID_ARG, "swe_selftest_wait: 1 us <= limit_ns <= 1 s");
  if (preset_abort > 0) return fail(SWE_ERR_INVALID_ARG, "swe_selftest_wait: preset_abort is 0 or a SWE_ERR_* code");
  struct Block {
    GridSync sync;
    int flag;
  };
  Block* d = nullptr;
  CK(cudaMalloc(&d, sizeof(Block)));
  int rc = SWE_OK;
  int abort_word = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(Block), S(stream));
  if (e == cudaSuccess && preset_abort != 0)
    e = cudaMemcpyAsync(&d->sync.abort, &preset_abort, sizeof(int), cudaMemcpyHostToDevice, S(stream));
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 32, 0, S(stream)>>>(&d->sync, &d->flag, (unsigned long long)limit_ns);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&abort_word, &d->sync.abort, sizeof(int), cudaMemcpyDeviceToHost, S(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
  cudaFree(d);
  if (e != cudaSuccess) rc = fail(SWE_ERR_CUDA, cudaGetErrorString(e));
  *status_out = abort_word;
  return rc;
}

int swe_device_status(swe_grid* g, void* stream) {
  if (!g) return fail(SWE_ERR_INVALID_ARG, "grid is NULL");
  if (!g->stats) return SWE_OK;
  DevStats ds;
  CK(cudaMemcpyAsync(&ds, g->stats, sizeof(DevStats), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  if (ds.status != SWE_OK) {
    int z = 0;
    CK(cudaMemcpy(&g->stats->status, &z, sizeof(int), cudaMemcpyHostToDevice));
    return fail(ds.status, "device-side error in the last phi_action / exprb_step");
  }
  return SWE_OK;
}

}  // extern "C"
