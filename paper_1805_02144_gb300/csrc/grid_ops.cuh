// Persistent-kernel building blocks shared by the phipm_simul_iom2 launch and
// its adjoint: per-block cell ranges, fixed-order block sums, bounded grid
// barriers and grid reductions.  A (launch arguments) provides part (at
// least NRED x gn doubles), ctrl, sync and prof; SH (the kernel's
// shared-memory struct) provides gb, gn, t_last, red and ok; ctrl's type
// provides red[].
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
// Reductions in a fixed order.  An FP64 add has a dependent latency of about
// 64 cycles on this part (a shuffle plus add about 100), so the sums over
// blocks below load their operands together and add them as trees of fixed
// shape; the shape depends only on the launch (threads per block, blocks), so
// results are reproducible.
// ---------------------------------------------------------------------------

// In-place pairwise tree over q[0..S) (S a power of two): q[0] = the total.
template <int S, int K>
__device__ __forceinline__ void pair_tree(double (&q)[S][K]) {
#pragma unroll
  for (int w = S / 2; w >= 1; w >>= 1)
#pragma unroll
    for (int s = 0; s < w; ++s)
#pragma unroll
      for (int k = 0; k < K; ++k) q[s][k] = q[2 * s][k] + q[2 * s + 1][k];
}

// Sum of p[b * stride] over b in [0, n): chunks of eight consecutive b, each
// loaded together and added as a pairwise tree, chunk totals added in order.
__device__ __forceinline__ double sum_strided(const double* p, size_t stride, int n) {
  double t = 0.0;
  for (int b0 = 0; b0 < n; b0 += 8) {
    double q[8][1];
#pragma unroll
    for (int s = 0; s < 8; ++s) q[s][0] = b0 + s < n ? __ldcg(p + (size_t)(b0 + s) * stride) : 0.0;
    pair_tree(q);
    t += q[0][0];
  }
  return t;
}

// Block totals of K per-thread values: a shuffle tree in every warp, then
// thread 0 adds the warp totals in warp order (a short serial chain: a tree
// here costs registers that the 64-register FP32 variants spill).  Thread 0
// holds the totals on return.
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

// Totals over gn blocks of K values (value k of block b at part[k * gn + b]),
// by one warp: lane l takes blocks l, l + 32, ... in chunks whose loads are
// issued together and added as a pairwise tree, then a shuffle tree.  Lane 0
// holds the totals on return.
template <int K>
__device__ __forceinline__ void warp_sum_blocks(const double* part, int gn, double (&t)[K]) {
  constexpr int S = K <= 2 ? 8 : (K <= 4 ? 4 : 1);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < K; ++k) t[k] = 0.0;
  for (int b0 = lane; b0 < gn; b0 += 32 * S) {
    double q[S][K];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int b = b0 + 32 * s;
#pragma unroll
      for (int k = 0; k < K; ++k) q[s][k] = b < gn ? __ldcg(part + (size_t)k * gn + b) : 0.0;
    }
    pair_tree(q);
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] += q[0][k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
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
    sh.ok = flip_barrier(a.sync, sh.gb, sh.gn, SWE_ERR_TIMEOUT);
    phase_tick(a, sh, phase);
  }
  __syncthreads();
  return sh.ok;
}

// Grid reduction of K per-thread partials, then a barrier.  Each block sums
// its threads (block_sum) and publishes its totals (value k of block b at
// part[k * gn + b]); warp 0 of the block that arrives last sums them over
// blocks (warp_sum_blocks: a fixed order, so the result is reproducible),
// stores them in ctrl->red[], runs post(ctrl, true, sums) on its lane 0 (the
// sums passed in registers, so the post reads nothing back over the bus) and
// publishes; the other blocks wait for the publication.
// The K sums of a grid reduction, handed to the post function by value.
template <int K>
struct RedSums {
  double v[K];
  __device__ __forceinline__ double operator[](int k) const { return v[k]; }
};

template <int K, class A, class SH, class Post>
__device__ bool grid_reduce(const A& a, SH& sh, double (&v)[K], int phase, Post post) {
  static_assert(K <= NRED, "reduction width");
  block_sum<K>(v, sh.red);
  if (threadIdx.x < 32) {
    GridSync* s = a.sync;
    const int gn = sh.gn;
    unsigned int lastu = 0, g0 = 0;
    if (threadIdx.x == 0) {
      for (int k = 0; k < K; ++k) a.part[(size_t)k * gn + sh.gb] = v[k];
      g0 = *(volatile unsigned int*)&s->rgen;  // cannot advance before this block arrives
      bool last;
      flip_arrive(s, sh.gb, gn, &last);
      lastu = last ? 1u : 0u;
    }
    lastu = __shfl_sync(0xffffffffu, lastu, 0);
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    if (lastu) {
      __threadfence();
      double t[K];
      warp_sum_blocks<K>(a.part, gn, t);
      if (threadIdx.x == 0) {
        auto* vc = make_volatile(a.ctrl);
        RedSums<K> r;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          vc->red[k] = t[k];
          r.v[k] = t[k];
        }
        post(vc, true, r);
        __threadfence();
        *(volatile unsigned int*)&s->rgen = g0 + 1;
        sh.ok = ld_volatile_int(&s->abort) == 0;
      }
    } else if (threadIdx.x == 0) {
      const volatile unsigned int* rg = &s->rgen;
      const bool ok = bounded_spin(s, SWE_ERR_TIMEOUT, [&] { return *rg == g0; });
      __threadfence();
      sh.ok = ok && ld_volatile_int(&s->abort) == 0;
    }
    if (threadIdx.x == 0) phase_tick(a, sh, phase);
  }
  __syncthreads();
  return sh.ok;
}

// Grid reduction of nv <= blockDim.x values whose block totals thread 0 of
// every block has stored at partw[gb * WIDE_STRIDE + r].  Threads r < nv of
// the block that arrives last each sum value r over blocks (sum_strided)
// into ctrl->wide[r]; its thread 0 runs post(ctrl) and publishes; the other
// blocks wait for the publication.
template <class A, class SH, class Post>
__device__ bool grid_reduce_wide(const A& a, SH& sh, int nv, int phase, Post post) {
  __syncthreads();
  GridSync* s = a.sync;
  __shared__ unsigned int w_last, w_g0;
  if (threadIdx.x == 0) {
    w_g0 = *(volatile unsigned int*)&s->rgen;  // cannot advance before this block arrives
    bool last;
    flip_arrive(s, sh.gb, sh.gn, &last);
    w_last = last ? 1u : 0u;
    if (last) __threadfence();
  }
  __syncthreads();
  if (w_last) {
    if ((int)threadIdx.x < nv) {
      const double t = sum_strided(a.partw + threadIdx.x, WIDE_STRIDE, sh.gn);
      ((volatile double*)a.ctrl->wide)[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence_block();
      post(make_volatile(a.ctrl));
      __threadfence();
      *(volatile unsigned int*)&s->rgen = w_g0 + 1;
      sh.ok = ld_volatile_int(&s->abort) == 0;
    }
  } else if (threadIdx.x == 0) {
    const volatile unsigned int* rg = &s->rgen;
    const unsigned int g0 = w_g0;
    const bool ok = bounded_spin(s, SWE_ERR_TIMEOUT, [&] { return *rg == g0; });
    __threadfence();
    sh.ok = ok && ld_volatile_int(&s->abort) == 0;
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
