// gp_device.cuh -- device-side helpers of the SSCN kernels: inline PTX for
// mbarriers, bulk (1D) copies and TMA tiled (3D) copies on sm_103a, bounded waits,
// the small real / complex arithmetic, and the field policies (pointwise substep,
// recurrence steps) shared by the sweeps and the standalone pointwise pass.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gp_internal.h"

namespace gpk {

// ------------------------------------------------------------------ bounds checks

// Built with -DGP_CHECK, GP_IN(i, n, status) is true when 0 <= i < n and otherwise
// records kStatusBounds in the solver's status word and is false, so that the access
// it guards is skipped (nothing traps; the host reports GP_ERR_BOUNDS).  In a normal
// build it is the constant true and the guarded code is unchanged.
#ifdef GP_CHECK
__device__ __forceinline__ bool check_index(long long i, long long n, int* status) {
  if (i >= 0 && i < n) return true;
  atomicOr(status, kStatusBounds);
  return false;
}
#define GP_IN(i, n, status) ::gpk::check_index((long long)(i), (long long)(n), (status))
#else
#define GP_IN(i, n, status) true
#endif

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of `bar`, giving up after `limit_ns` of wall time; a
// limit of 0 gives up at once (failure-detection tests).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (limit_ns == 0) return false;
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Contiguous global -> shared copy of `bytes` (multiple of 16, both ends 16-byte
// aligned); completion is signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Contiguous shared -> global copy, tracked by the bulk async-group.
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}

// 3D TMA tile load (coordinates in elements of the tensor map, x innermost).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// 3D TMA tile store; out-of-range parts of the box are not written.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2,
                                             const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          map),
      "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(src))
      : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the async proxy
// (TMA / bulk stores issued afterwards).
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 4- or 8-byte asynchronous global -> shared copy; fills zeros when !valid.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, bool valid) {
  const uint32_t n = valid ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_addr(dst)), "l"(src),
               "n"(BYTES), "r"(n)
               : "memory");
}
// 16-byte asynchronous global -> shared copy cached in L2 only; fills zeros when !valid
// (src must still be a valid address).
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool valid) {
  const uint32_t n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch: allow the next kernel of the stream to be scheduled
// (its blocks then wait in pdl_begin), and wait until the previous kernel has
// completed and its memory operations are visible.  Both are no-ops for a kernel
// launched without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// Wait for the tile's load (at most first_ns); on timeout flag it, then wait once
// more (at most kWaitLimitNs) so that no copy is left writing into shared memory
// after the block exits.
__device__ __forceinline__ bool wait_tile(uint64_t* bar, int* status, uint64_t first_ns) {
  if (mbar_wait_bounded(bar, 0, first_ns)) return true;
  if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
  mbar_wait_bounded(bar, 0, kWaitLimitNs);
  return false;
}

// ----------------------------------------------------- fused norm reduction

// Fixed-order block reduction of one FP64 value per warp into partials[block];
// the last block to finish sums the partials and writes the renormalisation factor.
// Every thread of the block must call it.  The last block's work is the kernel's
// tail (FP64 is narrow on this part: every dependent FP64 operation costs about a
// warp's worth of pipe cycles), so its sums are shallow pairwise trees in a fixed
// order: four partials per thread loaded together, (x0 + x1) + (x2 + x3), the warp
// shuffle tree, the warps' sums pairwise; the factor is rsqrt(norm), like
// 1 / sqrt(norm) within 1 ulp of the exact value.
__device__ __forceinline__ double sum_fixed(const double* w, int n) {
  if (n == 4) return (w[0] + w[1]) + (w[2] + w[3]);
  double v = w[0];
  for (int i = 1; i < n; ++i) v += w[i];
  return v;
}
__device__ __forceinline__ void norm_finish(double acc, double* partials, unsigned int* counter,
                                            unsigned int nb, unsigned int bid, double* scale_out,
                                            int* status, double dV) {
  __shared__ double wpart[kMaxBlockWarps];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) wpart[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    partials[bid] = sum_fixed(wpart, nw);
    // release of this block's partial and, for the last block, acquire of all the
    // others' (the counter's atomic updates form one release sequence); the block's
    // barrier then orders its threads' loads after the acquire
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(counter) : "memory");
    last = (old == nb - 1);
  }
  __syncthreads();
  if (!last) return;
  const unsigned int T = blockDim.x;
  auto quad = [&](unsigned int t0) {
    double x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned int t = t0 + q * T;
      x[q] = t < nb ? __ldcg(partials + t) : 0.0;
    }
    return (x[0] + x[1]) + (x[2] + x[3]);
  };
  double s = quad(threadIdx.x);
  for (unsigned int t0 = threadIdx.x + 4 * T; t0 < nb; t0 += 4 * T) s += quad(t0);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) wpart[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double norm = sum_fixed(wpart, nw) * dV;
    if (!(norm > 0.0) || !isfinite(norm)) atomicOr(status, kStatusNonFinite);
    *scale_out = rsqrt(norm);
    *counter = 0u;
  }
}

// Compensated FP32 pair (float-float): the value is hi + lo with |lo| <= ulp(hi) / 2.
// ff_add takes the error-free two-sum of the high parts (Knuth), adds the low parts to
// its error and renormalises: about 2^-44 relative error per addition, all on the
// FP32 pipe.  The FP32 sweeps sum their renormalisation norm this way: FP64 is narrow
// on this part, and a dependent FP64 tree at the end of every block held the z sweep
// back by about 4 us at 240 x 200 x 160.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bv = s - a.hi;
  const float e = ((a.hi - (s - bv)) + (b.hi - bv)) + (a.lo + b.lo);
  const float hi = s + e;
  return FF{hi, e - (hi - s)};
}
__device__ __forceinline__ FF ff_shfl_down(FF v, int o) {
  return FF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}

// norm_finish with the block's sums in float-float: every thread's FF value is summed
// in a fixed order (warp shuffle tree, warps in order) into partials[bid] (one FF per
// block, stored as a float pair); the last block to finish sums the nb partials in a
// fixed order over its threads, then in FP64 forms norm = (hi + lo) dV and writes the
// factor 1 / sqrt(norm).  With G > 1 the blocks take their tickets on G group counters
// (block b on gcounter[b mod G]) and only the last block of each group on `counter`:
// hundreds of blocks finishing together otherwise queue on one address at the L2.
// The acquire-release tickets chain, so the last block sees every partial.  The last
// block resets every counter it used.
// wpart_ff: shared memory for kMaxBlockWarps FF values and one int (a kernel may pass
// dynamic shared memory it no longer needs, behind a barrier).
__device__ __forceinline__ void norm_finish_ff(FF acc, FF* partials, unsigned int* counter,
                                               unsigned int nb, unsigned int bid, double* scale_out,
                                               int* status, double dV, unsigned int* gcounter,
                                               int G, FF* wpart_ff) {
  int& last_ff = *reinterpret_cast<int*>(wpart_ff + kMaxBlockWarps);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) acc = ff_add(acc, ff_shfl_down(acc, o));
  if (lane == 0) wpart_ff[warp] = acc;
  __syncthreads();
  const unsigned int ngroups = G > 1 ? min((unsigned int)G, nb) : 1u;
  if (threadIdx.x == 0) {
    FF b = wpart_ff[0];
    for (int w = 1; w < nw; ++w) b = ff_add(b, wpart_ff[w]);
    partials[bid] = b;
    // release of this block's partial and, for the last block, acquire of all the
    // others' (see norm_finish)
    bool last = false;
    if (G > 1) {
      const unsigned int g = bid % (unsigned int)G;
      const unsigned int gsize = (nb - g + G - 1) / G;   // blocks b < nb with b mod G == g
      if (atom_add_acq_rel(gcounter + g) == gsize - 1) last = atom_add_acq_rel(counter) == ngroups - 1;
    } else {
      last = atom_add_acq_rel(counter) == nb - 1;
    }
    last_ff = last;
  }
  __syncthreads();
  if (!last_ff) return;
  // a thread's partials t, t + T, ... are loaded eight at a time, all in flight
  // together (one L2 round trip per eight, not per partial), then added in order
  FF s = FF{0.f, 0.f};
  const unsigned int T = blockDim.x;
  for (unsigned int t0 = threadIdx.x; t0 < nb; t0 += 8 * T) {
    float2 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const unsigned int t = t0 + q * T;
      v[q] = t < nb ? __ldcg(reinterpret_cast<const float2*>(partials) + t) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s = ff_add(s, FF{v[q].x, v[q].y});
  }
  for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_down(s, o));
  if (lane == 0) wpart_ff[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    FF b = wpart_ff[0];
    for (int w = 1; w < nw; ++w) b = ff_add(b, wpart_ff[w]);
    const double norm = ((double)b.hi + (double)b.lo) * dV;
    if (!(norm > 0.0) || !isfinite(norm)) atomicOr(status, kStatusNonFinite);
    *scale_out = rsqrt(norm);
    *counter = 0u;
  }
  if (G > 1)
    for (unsigned int g = threadIdx.x; g < ngroups; g += blockDim.x) gcounter[g] = 0u;
}

// Fixed-order block sum of the nb float-float partials of a deferred norm, the same
// bits in every block of every kernel that takes it: thread t adds partials t, t + T,
// ... (all its loads in flight together), then the warp shuffle tree, then the warps
// in order.  Every thread of the block must call it; all get the factor
// 1 / sqrt(dV sum), formed in FP32 (it scales an FP32 field; rsqrtf is within 2 ulp,
// and the factor is remeasured every step, so its error does not accumulate), and the
// block's thread 0 flags a non-finite or zero norm when flag is set.
__device__ __forceinline__ double deferred_scale(const double* partials, int nb, double dV,
                                                 int* status, bool flag, const int* state = nullptr,
                                                 const double* stored = nullptr) {
  __shared__ FF wsum[kMaxBlockWarps];
  __shared__ double result;
  // with `state`: the partials are read whatever it holds (they are always valid memory)
  // so that its load and theirs are in flight together; the result is the partials'
  // factor when *state is 1 and *stored otherwise
  const int st = state ? *state : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned int T = blockDim.x;
  FF s = FF{0.f, 0.f};
  for (unsigned int t0 = threadIdx.x; t0 < (unsigned int)nb; t0 += 8 * T) {
    float2 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const unsigned int t = t0 + q * T;
      v[q] = t < (unsigned int)nb ? __ldcg(reinterpret_cast<const float2*>(partials) + t)
                                  : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s = ff_add(s, FF{v[q].x, v[q].y});
  }
  for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_down(s, o));
  if (lane == 0) wsum[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    FF b = wsum[0];
    for (int w = 1; w < nw; ++w) b = ff_add(b, wsum[w]);
    const float norm = (b.hi + b.lo) * (float)dV;
    if (st) {
      if (flag && (!(norm > 0.f) || !isfinite(norm))) atomicOr(status, kStatusNonFinite);
      result = (double)rsqrtf(norm);
    } else {
      result = *stored;
    }
  }
  __syncthreads();
  return result;
}

// ------------------------------------------------------------------- arithmetic

template <class R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };

__device__ __forceinline__ double gp_exp(double x) { return exp(x); }
__device__ __forceinline__ float gp_exp(float x) { return expf(x); }
__device__ __forceinline__ void gp_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void gp_sincos(float x, float* s, float* c) { sincosf(x, s, c); }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }

// a * b + c for complex a, b, c
template <class C> __device__ __forceinline__ C cfma(C a, C b, C c) {
  C r;
  r.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
  r.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
  return r;
}

template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

// ----------------------------------------------------------- field policies

// Dither of the renormalisation factor of an FP32 field in imaginary time: step n
// applies s (1 + xi_n 2^-20), xi_n = (int)(n 0x9E3779B9) / 2^31 in [-1, 1) (a Weyl
// sequence of the golden ratio, equidistributed).  At the ground state the FP32 field
// barely changes from step to step, so without it every step would round the same
// values the same way: a fixed error vector, which imaginary time amplifies by
// 1 / (dt gap) (about 500 at dt = 0.001).  A factor that moves the values by a few
// ulps per step turns that into zero-mean noise, which the step damps; the uniform
// factor itself is removed by the next renormalisation.  ctr = null: no dither.
__device__ __forceinline__ double step_dither(const unsigned int* ctr) {
  if (!ctr) return 1.0;
  const unsigned int u = *ctr * 0x9E3779B9u;
  return 1.0 + (double)(int)u * 0x1p-51;
}
// The same factor in FP32 (its steps of 2^-23 near 1), for kernels whose every thread
// forms the factor: no FP64 arithmetic, which is slow on this part.
__device__ __forceinline__ float step_dither_f(const unsigned int* ctr) {
  if (!ctr) return 1.f;
  const unsigned int u = *ctr * 0x9E3779B9u;
  return 1.f + (float)(int)u * 0x1p-51f;
}

template <class R, bool CPLX> struct Field;

// Real field, imaginary time.
template <class R> struct Field<R, false> {
  using E = R;
  static __device__ __forceinline__ E zero() { return R(0); }
  static __device__ __forceinline__ E scaled(E v, R s) { return v * s; }
  // v exp(-dt (V + g v^2))
  static __device__ __forceinline__ E pointwise(E v, R V, R dt, R g) {
    return v * gp_exp(-dt * fma(g * v, v, V));
  }
  // off-chain part of the forward step: A v_j + B (v_{j-1} + v_{j+1})
  static __device__ __forceinline__ E rhs(E A, E B, E prev, E next, E cur) {
    return fma(B, prev + next, A * cur);
  }
  static __device__ __forceinline__ E chain(E B, E x, E c) { return fma(B, x, c); }
  static __device__ __forceinline__ E mul(E a, E b) { return a * b; }
  static __device__ __forceinline__ E add(E a, E b) { return a + b; }
  static __device__ __forceinline__ R abs2(E v) { return v * v; }
  // v f exp(-y) with f = exp(-dt V) from the separable trap tables and y = dt g v^2:
  // for |y| <= 1/16 exp(-y) by its Taylor polynomial, of degree 4 in FP32 (remainder
  // below |y|^5/120 < 1e-8, under FP32 rounding) and 9 in FP64 (below |y|^10/10! <
  // 3e-19, under FP64 rounding), else by the library exp
  static __device__ __forceinline__ E nonlinear_small(E v, E f, R y) {
    const R z = -y;
    R q;
    if constexpr (sizeof(R) == 8) {
      q = fma(z, R(1.0 / 362880.0), R(1.0 / 40320.0));
      q = fma(z, q, R(1.0 / 5040.0));
      q = fma(z, q, R(1.0 / 720.0));
      q = fma(z, q, R(1.0 / 120.0));
      q = fma(z, q, R(1.0 / 24.0));
      q = fma(z, q, R(1.0 / 6.0));
    } else {
      q = fma(z, R(1.0 / 24.0), R(1.0 / 6.0));
    }
    q = fma(z, q, R(0.5));
    q = fma(z, q, R(1));
    q = fma(z, q, R(1));
    return v * f * q;
  }
  static __device__ __forceinline__ E nonlinear_full(E v, E f, R y) { return v * f * gp_exp(-y); }
};

// Complex field, real time.
template <class R> struct Field<R, true> {
  using E = typename Cplx<R>::T;
  static __device__ __forceinline__ E zero() { return E{R(0), R(0)}; }
  static __device__ __forceinline__ E scaled(E v, R s) { return E{v.x * s, v.y * s}; }
  // v exp(-i dt (V + g |v|^2)) = v (cos th - i sin th)
  static __device__ __forceinline__ E pointwise(E v, R V, R dt, R g) {
    const R th = dt * fma(g, fma(v.x, v.x, v.y * v.y), V);
    R sn, cs;
    gp_sincos(th, &sn, &cs);
    return E{fma(v.x, cs, v.y * sn), fma(v.y, cs, -v.x * sn)};
  }
  static __device__ __forceinline__ E rhs(E A, E B, E prev, E next, E cur) {
    return cfma(B, cadd(prev, next), cmul(A, cur));
  }
  static __device__ __forceinline__ E chain(E B, E x, E c) { return cfma(B, x, c); }
  static __device__ __forceinline__ E mul(E a, E b) { return cmul(a, b); }
  static __device__ __forceinline__ E add(E a, E b) { return cadd(a, b); }
  static __device__ __forceinline__ R abs2(E v) { return fma(v.x, v.x, v.y * v.y); }
  // v f (cos th - i sin th) with f = cis(-dt V) from the separable trap tables and
  // th = dt g |v|^2: for |th| <= 1/16 cos and sin by their Taylor polynomials, of
  // degrees 4 and 5 in FP32 (remainders below th^6/720 and th^7/5040) and 8 and 9 in
  // FP64 (below th^10/10! and th^11/11!), else the library sincos
  static __device__ __forceinline__ E nonlinear_small(E v, E f, R th) {
    const R t2 = th * th;
    R cs, sn;
    if constexpr (sizeof(R) == 8) {
      cs = fma(t2, R(1.0 / 40320.0), R(-1.0 / 720.0));
      cs = fma(t2, cs, R(1.0 / 24.0));
      sn = fma(t2, R(1.0 / 362880.0), R(-1.0 / 5040.0));
      sn = fma(t2, sn, R(1.0 / 120.0));
    } else {
      cs = R(1.0 / 24.0);
      sn = R(1.0 / 120.0);
    }
    cs = fma(t2, fma(t2, cs, R(-0.5)), R(1));
    sn = th * fma(t2, fma(t2, sn, R(-1.0 / 6.0)), R(1));
    return cmul(cmul(v, f), E{cs, -sn});
  }
  static __device__ __forceinline__ E nonlinear_full(E v, E f, R th) {
    R sn, cs;
    gp_sincos(th, &sn, &cs);
    return cmul(cmul(v, f), E{cs, -sn});
  }
};

}  // namespace gpk
