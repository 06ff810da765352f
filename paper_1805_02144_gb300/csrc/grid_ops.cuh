// Persistent-kernel building blocks shared by the phipm_simul_iom2 launch and
// its adjoint: per-block cell ranges, fixed-order block sums, bounded grid
// barriers and grid reductions.  A (launch arguments) provides part, ctrl,
// sync and prof; SH (the kernel's shared-memory struct) provides gb, gn,
// t_last, red, gen, last and ok; ctrl's type provides red[].
#pragma once
#include <cuda_runtime.h>

#include "../../include/swe_exprb.h"
#include "phi_args.h"
#include "swe_dev.cuh"

namespace swe {

template <class C>
__device__ __forceinline__ volatile C* make_volatile(C* p) { return p; }

__device__ __forceinline__ double vld(const double* p) { return *(volatile const double*)p; }
__device__ __forceinline__ int vldi(const int* p) { return *(volatile const int*)p; }

struct Range {
  int c0, c1;
};

// Cells of this thread inside the block's range (block-strided).
struct CellLoop {
  int first, end, step;
  __device__ CellLoop(const Range& R) {
    first = R.c0 + threadIdx.x;
    end = R.c1;
    step = blockDim.x;
  }
};
#define FOR_CELLS(i) for (int i = CL.first; i < CL.end; i += CL.step)

// ---------------------------------------------------------------------------
// block reductions in a fixed order
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sred[warp * NRED + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w * NRED + k];
      v[k] = s;
    }
  }
  __syncthreads();
}

template <class A, class SH>
__device__ __forceinline__ void phase_tick(const A& a, SH& sh, int phase) {
  if (a.prof && sh.gb == 0 && threadIdx.x == 0) {
    unsigned long long now = globaltimer();
    a.prof->phase_ns[phase] += (long long)(now - sh.t_last);
    sh.t_last = now;
  }
}

// Plain grid barrier.  Returns false (uniformly per block) when the launch is
// being aborted.
template <class A, class SH>
__device__ bool grid_barrier(const A& a, SH& sh, int phase) {
  __syncthreads();
  if (threadIdx.x == 0) {
    bool last;
    unsigned int gen = bar_arrive(a.sync, sh.gn, &last);
    bool ok = true;
    if (last)
      bar_release(a.sync, gen);
    else
      ok = bar_wait(a.sync, gen, SWE_ERR_TIMEOUT);
    sh.ok = ok && (ld_volatile_int(&a.sync->abort) == 0);
    phase_tick(a, sh, phase);
  }
  __syncthreads();
  return sh.ok;
}

// Grid reduction of K per-thread partials, then a barrier.  The last block
// to arrive sums the block partials in block order, stores them in
// ctrl->red[], runs post(ctrl) on its thread 0, and releases the barrier.
template <int K, class A, class SH, class Post>
__device__ bool grid_reduce(const A& a, SH& sh, double (&v)[K], int phase, Post post) {
  block_sum<K>(v, sh.red);
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) a.part[(size_t)sh.gb * NRED + k] = v[k];
    bool last;
    sh.gen = bar_arrive(a.sync, sh.gn, &last);
    sh.last = last;
  }
  __syncthreads();
  if (sh.last) {
    double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int b = threadIdx.x; b < sh.gn; b += blockDim.x) s += a.part[(size_t)b * NRED + k];
      tot[k] = s;
    }
    block_sum<K>(tot, sh.red);
    if (threadIdx.x == 0) {
      auto* vc = make_volatile(a.ctrl);
      for (int k = 0; k < K; ++k) vc->red[k] = tot[k];
      post(vc);
      bar_release(a.sync, sh.gen);
      sh.ok = ld_volatile_int(&a.sync->abort) == 0;
    }
  } else if (threadIdx.x == 0) {
    bool ok = bar_wait(a.sync, sh.gen, SWE_ERR_TIMEOUT);
    sh.ok = ok && (ld_volatile_int(&a.sync->abort) == 0);
  }
  if (threadIdx.x == 0) phase_tick(a, sh, phase);
  __syncthreads();
  return sh.ok;
}

template <class A>
__device__ __forceinline__ void abort_launch(const A& a, int code) {
  atomicCAS(&a.sync->abort, 0, code);
}

}  // namespace swe
