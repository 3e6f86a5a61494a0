// gp_reduce.cu -- one-pass FP64 reductions and field conversions around the SSCN
// step: observables (energy, chemical potential, rms sizes), the norm of a fresh
// state, the initial Gaussian, host-layout import / export, and the integrated
// densities of Eq. 1 and its 3D analogues (paper, "Summary of revisions").
//
// Every reduction runs on a fixed launch shape (kReduceBlocks x kReduceThreads),
// sums in a fixed order (per thread, then a shuffle tree, then the blocks' partials
// in index order by the last block to finish), and is therefore deterministic.
#include "gp_device.cuh"

namespace gpk {

template <class R, bool CPLX> struct Load;
template <class R> struct Load<R, false> {
  static __device__ __forceinline__ double2 at(const void* psi, size_t idx, double s) {
    return make_double2((double)static_cast<const R*>(psi)[idx] * s, 0.0);
  }
};
template <class R> struct Load<R, true> {
  static __device__ __forceinline__ double2 at(const void* psi, size_t idx, double s) {
    const typename Cplx<R>::T v = static_cast<const typename Cplx<R>::T*>(psi)[idx];
    return make_double2((double)v.x * s, (double)v.y * s);
  }
};

__device__ __forceinline__ double dabs2(double2 v) { return fma(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ double dabs2_diff(double2 a, double2 b) {
  const double x = a.x - b.x, y = a.y - b.y;
  return fma(x, x, y * y);
}

// Fixed-order block sum of NACC accumulators into partials[blockIdx.x * NACC + c];
// returns true in the last block to finish, after its fixed-order total over all
// blocks has been written to tot[0..NACC-1] (shared memory).  Every thread of every
// block must call it.
template <int NACC>
__device__ bool block_reduce_last(double (&acc)[NACC], double* partials, unsigned int* counter,
                                  double* tot) {
  __shared__ double warp_part[kReduceThreads / 32][NACC];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NACC; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) warp_part[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < NACC) {
    double v = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) v += warp_part[w][threadIdx.x];
    partials[(size_t)blockIdx.x * NACC + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // the blocks' partials of each accumulator: thread t takes blocks t, t + T, ...
  // (Neumaier), then a shuffle tree and the warps in order -- a fixed order, and
  // short FP64 dependency chains (one thread walking all blocks would take a chain
  // of four FP64 operations per block)
  const unsigned int nb = gridDim.x;
#pragma unroll
  for (int c = 0; c < NACC; ++c) {
    double s = 0.0, comp = 0.0;
    for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x) {
      const double x = __ldcg(partials + (size_t)b * NACC + c);
      const double u = s + x;
      comp += (fabs(s) >= fabs(x)) ? (s - u) + x : (x - u) + s;
      s = u;
    }
    double v = s + comp;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) warp_part[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < NACC) {
    double v = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) v += warp_part[w][threadIdx.x];
    tot[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ---------------------------------------------------------------- observables

template <class R, bool CPLX>
__global__ void __launch_bounds__(kReduceThreads) k_observables(const FieldParams p) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const size_t P = (size_t)p.pitch, plane = P * ny;
  const double s = *p.scale;
  const double* Vx = p.tab;
  const double* Vy = Vx + nx;
  const double* Vz = Vy + ny;
  const double* X2 = Vz + nz;
  const double* Y2 = X2 + nx;
  const double* Z2 = Y2 + ny;
  double acc[kObsAcc];
#pragma unroll
  for (int c = 0; c < kObsAcc; ++c) acc[c] = 0.0;
  const long long nrows = (long long)ny * nz;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const size_t base = (size_t)r * P;
    const double vyz = Vy[j] + Vz[k];
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const size_t idx = base + i;
      const double2 v = Load<R, CPLX>::at(p.psi, idx, s);
      const double d = dabs2(v);
      acc[0] += d;
      acc[1] += (Vx[i] + vyz) * d;
      acc[2] += d * d;
      const double2 z0 = make_double2(0.0, 0.0);
      const double2 wx = (i + 1 < nx) ? Load<R, CPLX>::at(p.psi, idx + 1, s) : z0;
      const double2 wy = (j + 1 < ny) ? Load<R, CPLX>::at(p.psi, idx + P, s) : z0;
      const double2 wz = (k + 1 < nz) ? Load<R, CPLX>::at(p.psi, idx + plane, s) : z0;
      acc[3] += dabs2_diff(wx, v) + (i == 0 ? d : 0.0);  // edge (i, i+1), ghost edge at i = 0
      acc[4] += dabs2_diff(wy, v) + (j == 0 ? d : 0.0);
      acc[5] += dabs2_diff(wz, v) + (k == 0 ? d : 0.0);
      acc[6] += X2[i] * d;
      acc[7] += Y2[j] * d;
      acc[8] += Z2[k] * d;
    }
  }
  __shared__ double tot[kObsAcc];
  if (!block_reduce_last<kObsAcc>(acc, p.partials, p.counter, tot)) return;
  if (threadIdx.x == 0) {
    const double dV = p.hx * p.hy * p.hz;
    const double norm = tot[0] * dV;
    const double epot = tot[1] * dV;
    const double eint = 0.5 * p.g * tot[2] * dV;
    const double ekin =
        0.5 * dV * (tot[3] / (p.hx * p.hx) + tot[4] / (p.hy * p.hy) +
                    (p.nz == 1 ? 0.0 : tot[5] / (p.hz * p.hz)));   // 2D: no z kinetic term
    const double x2 = tot[6] * dV / norm, y2 = tot[7] * dV / norm, z2 = tot[8] * dV / norm;
    double* o = p.out;
    o[0] = norm;
    o[1] = ekin + epot + 2.0 * eint;
    o[2] = ekin + epot + eint;
    o[3] = ekin;
    o[4] = epot;
    o[5] = eint;
    o[6] = sqrt(x2);
    o[7] = sqrt(y2);
    o[8] = sqrt(z2);
    o[9] = sqrt(x2 + y2 + z2);
  }
}

// ------------------------------------------------------ norm of a fresh field

// Real field only (used after the Gaussian initialisation): *out = 1/sqrt(norm).
template <class R>
__global__ void __launch_bounds__(kReduceThreads) k_norm_to_scale(const FieldParams p) {
  const int nx = p.nx;
  const size_t P = (size_t)p.pitch;
  double acc[1] = {0.0};
  const long long nrows = (long long)p.ny * p.nz;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = (double)static_cast<const R*>(p.psi)[(size_t)r * P + i];
      acc[0] += v * v;
    }
  __shared__ double tot[1];
  if (!block_reduce_last<1>(acc, p.partials, p.counter, tot)) return;
  if (threadIdx.x == 0) {
    const double norm = tot[0] * p.hx * p.hy * p.hz;
    if (!(norm > 0.0) || !isfinite(norm)) atomicOr(p.status, kStatusNonFinite);
    *p.out = 1.0 / sqrt(norm);
  }
}

// ------------------------------------------- standalone pointwise substep

// psi <- P(psi) with the half step's separable trap factors and dtg = (dt / 2) g, the
// same arithmetic as the sweeps' fused substep (Field policies); with NORM the norm
// of the result becomes the pending factor.
template <class R, bool CPLX, bool NORM>
__global__ void __launch_bounds__(kReduceThreads) k_half_pointwise(const FieldParams p, const void* fx,
                                                                   const void* fyz, double dtg_d,
                                                                   int apply_scale) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  const int nx = p.nx;
  const size_t P = (size_t)p.pitch;
  const R s = apply_scale ? (R)(*p.scale) : R(1);
  const R dtg = (R)dtg_d;
  const E* fxt = static_cast<const E*>(fx);
  const E* fyt = static_cast<const E*>(fyz);
  E* psi = static_cast<E*>(p.psi);
  double acc[1] = {0.0};
  // chunks of CH rows, the chunk's CH * nx points spread over the block, U per thread
  // in flight: all U loads are issued before any store
  constexpr int U = 4, CH = 8;
  const long long nrows = (long long)p.ny * p.nz;
  const int per = CH * nx;   // points per chunk
  for (long long r0 = (long long)blockIdx.x * CH; r0 < nrows; r0 += (long long)gridDim.x * CH) {
    const int rows = (int)min((long long)CH, nrows - r0);
    const int cnt = rows * nx;
    for (int base = threadIdx.x; base < cnt; base += blockDim.x * U) {
      E v[U], f[U];
      size_t at[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * blockDim.x;
        const int q = e < cnt ? e : 0;
        const int rl = q / nx, i = q - rl * nx;
        at[u] = (size_t)(r0 + rl) * P + i;
        v[u] = psi[at[u]];
        f[u] = F::mul(fxt[i], fyt[r0 + rl]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (base + u * (int)blockDim.x >= cnt) continue;
        const E w = F::scaled(v[u], s);
        const R y = dtg * F::abs2(w);
        const E out = fabs(y) <= R(0.0625) ? F::nonlinear_small(w, f[u], y) : F::nonlinear_full(w, f[u], y);
        psi[at[u]] = out;
        if (NORM) acc[0] += (double)F::abs2(out);
      }
    }
    (void)per;
  }
  if (NORM) {
    __shared__ double tot[1];
    if (!block_reduce_last<1>(acc, p.partials, p.counter, tot)) return;
    if (threadIdx.x == 0) {
      const double norm = tot[0] * p.hx * p.hy * p.hz;
      if (!(norm > 0.0) || !isfinite(norm)) atomicOr(p.status, kStatusNonFinite);
      *p.out = 1.0 / sqrt(norm);
    }
  }
}

// FP32 field (words = 1 real, 2 complex floats per element) times the pending factor,
// packed into rows of nx elements in dst (not the field): 16-byte vectors when the
// rows are contiguous and a multiple of four floats, else one float per thread.
__global__ void k_export_f32(const FieldParams p, int words, float* __restrict__ dst) {
  const float s = (float)(*p.scale);
  const float* src = static_cast<const float*>(p.psi);
  const size_t rw = (size_t)p.nx * words, pw = (size_t)p.pitch * words;
  const size_t nrows = (size_t)p.ny * p.nz;
  if (rw == pw && rw % 4 == 0) {
    const size_t n4 = nrows * rw / 4;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
      float4 v = s4[i];
      v.x *= s;
      v.y *= s;
      v.z *= s;
      v.w *= s;
      d4[i] = v;
    }
    return;
  }
  for (size_t r = blockIdx.x; r < nrows; r += gridDim.x)
    for (size_t i = threadIdx.x; i < rw; i += blockDim.x) dst[r * rw + i] = src[r * pw + i] * s;
}

// The reverse: packed rows of nx elements in src into the FP32 field (pad columns
// zero), as they are (no factor).
__global__ void k_import_f32(const FieldParams p, int words, const float* __restrict__ src) {
  float* dst = static_cast<float*>(p.psi);
  const size_t rw = (size_t)p.nx * words, pw = (size_t)p.pitch * words;
  const size_t nrows = (size_t)p.ny * p.nz;
  if (rw == pw && rw % 4 == 0) {
    const size_t n4 = nrows * rw / 4;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
      d4[i] = s4[i];
    return;
  }
  for (size_t r = blockIdx.x; r < nrows; r += gridDim.x)
    for (size_t i = threadIdx.x; i < pw; i += blockDim.x) dst[r * pw + i] = i < rw ? src[r * rw + i] : 0.f;
}

// ------------------------------------------------------------ initial Gaussian

template <class R>
__global__ void k_init_gaussian(const FieldParams p, double wx, double wy, double wz) {
  const int nx = p.nx, ny = p.ny, P = p.pitch;
  const long long nrows = (long long)ny * p.nz;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const double y = (j - 0.5 * (ny - 1)) * p.hy;
    const double z = (k - 0.5 * (p.nz - 1)) * p.hz;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      double v = 0.0;
      if (i < nx) {
        const double x = (i - 0.5 * (nx - 1)) * p.hx;
        v = exp(-0.5 * (wx * x * x + wy * y * y + wz * z * z));
      }
      static_cast<R*>(p.psi)[(size_t)r * P + i] = (R)v;
    }
  }
}

// ------------------------------------------------- host layout <-> device field

template <class R, bool CPLX>
__global__ void k_import(const FieldParams p, const double* __restrict__ src) {
  using C = typename Cplx<R>::T;
  const int nx = p.nx, P = p.pitch;
  const long long nrows = (long long)p.ny * p.nz;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x)
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      const size_t d = (size_t)r * P + i, q = (size_t)r * nx + i;
      if (CPLX) {
        C v{R(0), R(0)};
        if (i < nx) v = C{(R)src[2 * q], (R)src[2 * q + 1]};
        static_cast<C*>(p.psi)[d] = v;
      } else {
        static_cast<R*>(p.psi)[d] = i < nx ? (R)src[q] : R(0);
      }
    }
}

template <class R, bool CPLX>
__global__ void k_export(const FieldParams p, double* __restrict__ dst, int as_complex) {
  const int nx = p.nx;
  const size_t P = (size_t)p.pitch;
  const double s = *p.scale;
  const long long nrows = (long long)p.ny * p.nz;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double2 v = Load<R, CPLX>::at(p.psi, (size_t)r * P + i, s);
      const size_t q = (size_t)r * nx + i;
      if (as_complex) {
        dst[2 * q] = v.x;
        dst[2 * q + 1] = v.y;
      } else {
        dst[q] = v.x;
      }
    }
}

// ------------------------------------------------------- integrated densities

// plane 0: out[j*nx+i] = dz sum_k |psi|^2 ; plane 1: out[k*nx+i] = dy sum_j |psi|^2
template <class R, bool CPLX>
__global__ void k_density_sum_strided(const FieldParams p, int plane, double* __restrict__ out) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const size_t P = (size_t)p.pitch;
  const double s = *p.scale;
  const int rows = plane == 0 ? ny : nz;          // output rows
  const int nsum = plane == 0 ? nz : ny;          // summed extent
  const size_t step = plane == 0 ? P * ny : P;    // stride of the summed axis
  const double w = plane == 0 ? p.hz : p.hy;
  const long long total = (long long)rows * nx;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % nx), o = (int)(q / nx);
    const size_t base = plane == 0 ? (size_t)o * P + i : (size_t)o * P * ny + i;
    double acc = 0.0;
    for (int t = 0; t < nsum; ++t) acc += dabs2(Load<R, CPLX>::at(p.psi, base + t * step, s));
    out[q] = acc * w;
  }
}

// plane 2: out[k*ny+j] = dx sum_i |psi|^2, one warp per (j, k) row
template <class R, bool CPLX>
__global__ void k_density_sum_rows(const FieldParams p, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nrows = (long long)p.ny * p.nz;
  const double s = *p.scale;
  for (long long r = warp; r < nrows; r += nwarps) {
    double acc = 0.0;
    for (int i = lane; i < p.nx; i += 32)
      acc += dabs2(Load<R, CPLX>::at(p.psi, (size_t)r * p.pitch + i, s));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r] = acc * p.hx;
  }
}

// out[r] = w * sum_c in[r*cols + c], one warp per row
__global__ void k_rows_sum(const double* __restrict__ in, int rows, int cols, double w,
                           double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= rows) return;
  double acc = 0.0;
  for (int c = lane; c < cols; c += 32) acc += in[(size_t)warp * cols + c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = acc * w;
}

// out[c] = w * sum_r in[r*cols + c], one thread per column
__global__ void k_cols_sum(const double* __restrict__ in, int rows, int cols, double w,
                           double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double acc = 0.0;
  for (int r = 0; r < rows; ++r) acc += in[(size_t)r * cols + c];
  out[c] = acc * w;
}

// ---------------------------------------------------------------- launchers

static unsigned int grid_for_rows(const FieldParams& p) {
  const long long nrows = (long long)p.ny * p.nz;
  return (unsigned int)(nrows < 4096 ? nrows : 4096);
}

template <class R>
cudaError_t launch_observables(const FieldParams& p, bool complex_field, cudaStream_t st) {
  if (complex_field)
    k_observables<R, true><<<kReduceBlocks, kReduceThreads, 0, st>>>(p);
  else
    k_observables<R, false><<<kReduceBlocks, kReduceThreads, 0, st>>>(p);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_resolve_scale(double* scale, int* state, const double* partials,
                                                      int nb, double dV, int* status) {
  if (*state == 0) return;   // uniform: every thread reads the same word
  const double f = deferred_scale(partials, nb, dV, status, true);
  if (threadIdx.x == 0) {
    *scale = f;
    *state = 0;
  }
}

cudaError_t launch_resolve_scale(double* scale, int* state, const double* partials, int nb,
                                 double dV, int* status, cudaStream_t st) {
  k_resolve_scale<<<1, 256, 0, st>>>(scale, state, partials, nb, dV, status);
  return cudaGetLastError();
}

template <class R> cudaError_t launch_norm_to_scale(const FieldParams& p, cudaStream_t st) {
  k_norm_to_scale<R><<<kReduceBlocks, kReduceThreads, 0, st>>>(p);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_half_pointwise(const FieldParams& p, bool complex_field, const void* fx,
                                  const void* fyz, double dtg, bool apply_scale, bool norm,
                                  cudaStream_t st) {
  const int as = apply_scale ? 1 : 0;
  if (complex_field) {
    if (norm) k_half_pointwise<R, true, true><<<kReduceBlocks, kReduceThreads, 0, st>>>(p, fx, fyz, dtg, as);
    else k_half_pointwise<R, true, false><<<kReduceBlocks, kReduceThreads, 0, st>>>(p, fx, fyz, dtg, as);
  } else {
    if (norm) k_half_pointwise<R, false, true><<<kReduceBlocks, kReduceThreads, 0, st>>>(p, fx, fyz, dtg, as);
    else k_half_pointwise<R, false, false><<<kReduceBlocks, kReduceThreads, 0, st>>>(p, fx, fyz, dtg, as);
  }
  return cudaGetLastError();
}


cudaError_t launch_export_f32(const FieldParams& p, bool complex_field, float* dst, cudaStream_t st) {
  k_export_f32<<<grid_for_rows(p), 256, 0, st>>>(p, complex_field ? 2 : 1, dst);
  return cudaGetLastError();
}

cudaError_t launch_import_f32(const FieldParams& p, bool complex_field, const float* src, cudaStream_t st) {
  k_import_f32<<<grid_for_rows(p), 256, 0, st>>>(p, complex_field ? 2 : 1, src);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_init_gaussian(const FieldParams& p, double wx, double wy, double wz,
                                 cudaStream_t st) {
  k_init_gaussian<R><<<grid_for_rows(p), 256, 0, st>>>(p, wx, wy, wz);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_import(const FieldParams& p, const double* src, bool complex_field,
                          cudaStream_t st) {
  if (complex_field)
    k_import<R, true><<<grid_for_rows(p), 256, 0, st>>>(p, src);
  else
    k_import<R, false><<<grid_for_rows(p), 256, 0, st>>>(p, src);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_export(const FieldParams& p, double* dst, bool complex_field, bool as_complex,
                          cudaStream_t st) {
  if (complex_field)
    k_export<R, true><<<grid_for_rows(p), 256, 0, st>>>(p, dst, 1);
  else
    k_export<R, false><<<grid_for_rows(p), 256, 0, st>>>(p, dst, as_complex ? 1 : 0);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_density2d(const FieldParams& p, bool complex_field, int plane, double* out,
                             cudaStream_t st) {
  if (plane == 2) {
    if (complex_field)
      k_density_sum_rows<R, true><<<1024, 256, 0, st>>>(p, out);
    else
      k_density_sum_rows<R, false><<<1024, 256, 0, st>>>(p, out);
  } else {
    if (complex_field)
      k_density_sum_strided<R, true><<<1024, 256, 0, st>>>(p, plane, out);
    else
      k_density_sum_strided<R, false><<<1024, 256, 0, st>>>(p, plane, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_rows_sum(const double* in, int rows, int cols, double w, double* out,
                            cudaStream_t st) {
  const int threads = 256, warps_per_block = threads / 32;
  k_rows_sum<<<(rows + warps_per_block - 1) / warps_per_block, threads, 0, st>>>(in, rows, cols,
                                                                                  w, out);
  return cudaGetLastError();
}

cudaError_t launch_cols_sum(const double* in, int rows, int cols, double w, double* out,
                            cudaStream_t st) {
  k_cols_sum<<<(cols + 255) / 256, 256, 0, st>>>(in, rows, cols, w, out);
  return cudaGetLastError();
}

#define GP_INSTANTIATE(R)                                                                      \
  template cudaError_t launch_observables<R>(const FieldParams&, bool, cudaStream_t);         \
  template cudaError_t launch_norm_to_scale<R>(const FieldParams&, cudaStream_t);             \
  template cudaError_t launch_half_pointwise<R>(const FieldParams&, bool, const void*,       \
                                                const void*, double, bool, bool, cudaStream_t); \
  template cudaError_t launch_init_gaussian<R>(const FieldParams&, double, double, double,    \
                                               cudaStream_t);                                  \
  template cudaError_t launch_import<R>(const FieldParams&, const double*, bool, cudaStream_t); \
  template cudaError_t launch_export<R>(const FieldParams&, double*, bool, bool, cudaStream_t); \
  template cudaError_t launch_density2d<R>(const FieldParams&, bool, int, double*, cudaStream_t);
GP_INSTANTIATE(double)
GP_INSTANTIATE(float)
#undef GP_INSTANTIATE

}  // namespace gpk
