// swe_jv_noalloc: J(u) x without any device allocation.
//
// Who needs this: swe_jv sizes its scratch (the pass-1 planes and the
// eta / n x u planes of the linearisation state) inside the grid's workspace,
// which the library allocates with cudaMalloc on first use (and that workspace
// also holds the Krylov basis of phi_action).  Some callers must not allocate
// device memory at that point: code that runs under another framework's
// memory pool or under a fixed device-memory budget reserved at start-up
// (a cudaMalloc behind the pool's back breaks its accounting or fails), and
// real-time loops that cannot take an allocation's latency or an
// out-of-memory failure in the middle of a run.  This entry point uses a
// scratch array that is part of the library image instead.
//
// The scratch is one file-scope device array of kScratchDoubles doubles
// (12 planes of up to kMaxCells cells: 3.9 MB), resident on every GPU that
// loads the library until the process exits.  Its device address is looked up
// once per device with cudaGetSymbolAddress on the first call made with that
// device current; make that first call before any stream capture begins.
// Every call reuses the same array: each plane is fully written before it is
// read, so nothing needs clearing, but two calls that overlap on the GPU (for
// example on two streams) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/swe_exprb.h"
#include "swe_dev.cuh"

using namespace swe;

namespace swe {
// Device tables of a grid handle and the device they live on (defined with
// the handle in swe_api.cu).
int grid_device_tables(const swe_grid* g, Tables* out, int* device);
void set_last_error(const std::string& msg);
}  // namespace swe

namespace {

constexpr int kMaxCells = 40962;  // level-6 grid
constexpr size_t kScratchDoubles = (size_t)12 * kMaxCells;
static __device__ __align__(256) double g_jv_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

__global__ void k_aux_na(Tables T, const double* __restrict__ u, double* aux) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.ng; i += gridDim.x * blockDim.x)
    aux_cell(T, i, u, aux);
}

__global__ void k_pass1_na(Tables T, const double* x, const double* u, double* tmp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.ng; i += gridDim.x * blockDim.x)
    pass1_cell<MODE_J>(T, i, x, 1.0, u, tmp, tmp + (size_t)4 * T.ng);
}

__global__ void k_pass2_na(Tables T, const double* x, const double* tmp, const double* aux, double* out) {
  const int ng = T.ng;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
    double o[4];
    pass2_cell<MODE_J>(T, i, x, 1.0, tmp, tmp + (size_t)4 * ng, aux, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) out[(size_t)c * ng + i] = o[c];
  }
}

// Device address of the scratch array on device dev, which must be the
// current device (looked up once per device).
int scratch_ptr(int dev, double** out) {
  cudaError_t e;
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("swe_jv_noalloc: device ordinal out of range");
    return SWE_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_jv_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("swe_jv_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return SWE_ERR_CUDA;
    }
    g_ptr[dev] = (double*)p;
  }
  *out = g_ptr[dev];
  return SWE_OK;
}

}  // namespace

extern "C" int swe_jv_noalloc(const swe_grid* grid, const double* u, const double* x, double* jx,
                              void* stream) {
  if (!grid || !u || !x || !jx) {
    set_last_error("swe_jv_noalloc: NULL argument");
    return SWE_ERR_INVALID_ARG;
  }
  Tables T;
  int grid_dev = -1;
  int rc = grid_device_tables(grid, &T, &grid_dev);
  if (rc != SWE_OK) return rc;
  if (T.ng > kMaxCells) {
    set_last_error("swe_jv_noalloc: grid has " + std::to_string(T.ng) +
                   " cells; the static scratch holds at most " + std::to_string(kMaxCells) +
                   " (level 6); use swe_jv for larger grids");
    return SWE_ERR_INVALID_ARG;
  }
  // jx is written while neighbouring cells of x (and cell values of u) are
  // still being read: the output must not overlap either input
  const size_t nbytes = (size_t)4 * T.ng * sizeof(double);
  auto overlaps = [nbytes](const void* a, const void* b) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + nbytes && pb < pa + nbytes;
  };
  if (overlaps(jx, x) || overlaps(jx, u)) {
    set_last_error("swe_jv_noalloc: jx must not overlap u or x");
    return SWE_ERR_INVALID_ARG;
  }
  // the tables and the scratch belong to the grid's device: launching with
  // another device current would read the grid's memory from the wrong GPU
  int cur = -1;
  cudaError_t ge = cudaGetDevice(&cur);
  if (ge != cudaSuccess) {
    set_last_error(std::string("swe_jv_noalloc: cudaGetDevice: ") + cudaGetErrorString(ge));
    return SWE_ERR_CUDA;
  }
  if (cur != grid_dev) {
    set_last_error("swe_jv_noalloc: the grid was built on device " + std::to_string(grid_dev) +
                   " but device " + std::to_string(cur) + " is current");
    return SWE_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  if ((rc = scratch_ptr(cur, &scratch)) != SWE_OK) return rc;
  double* tmp = scratch;                          // 8 planes of ng
  double* aux = scratch + (size_t)8 * T.ng;       // 4 planes of ng
  cudaStream_t st = (cudaStream_t)stream;
  const int tpb = 256;
  int nb = (T.ng + tpb - 1) / tpb;
  k_aux_na<<<nb, tpb, 0, st>>>(T, u, aux);
  k_pass1_na<<<nb, tpb, 0, st>>>(T, x, u, tmp);
  k_pass2_na<<<nb, tpb, 0, st>>>(T, x, tmp, aux, jx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("swe_jv_noalloc: launch: ") + cudaGetErrorString(e));
    return SWE_ERR_CUDA;
  }
  return SWE_OK;
}
