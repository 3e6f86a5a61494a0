// gp_sweeps.cu -- the three Crank-Nicolson sweeps of one split-step Crank-Nicolson
// (SSCN) time step of the 3D Gross-Pitaevskii equation (paper, program summary:
// "Solution method"; imag3d / real3d summaries).
//
// One step with tau = dt (imaginary time, real field) or i dt (real time, complex
// field) is: the pointwise substep psi <- psi exp(-tau (V + g |psi|^2)), then a CN
// solve along every x line, every y line and every z line, then (imaginary time)
// renormalisation.  Each sweep is one kernel that reads and writes the field once:
//
//   sweep x  rows are contiguous, so a tile of W consecutive rows is one
//            contiguous block: one bulk copy (cp.async.bulk) brings it into shared
//            memory.  Before the solve each element gets the pending
//            renormalisation factor and the pointwise substep (fused on load).
//            Lane l solves row l; lanes walk their rows in a skewed wavefront
//            (lane l handles element t - l at step t when the pitch is even) so
//            that the 32 lanes always touch 32 different banks.
//   sweep y  a tile is W consecutive x positions times the whole y extent at one
//   sweep z  z (or W x positions times the whole z extent at one y), moved by 3D
//            TMA boxes.  Lane l solves the line at x = i0 + l; in shared memory
//            that line is a column, so the lanes are on consecutive words.
//            The z sweep, last of the step, also sums |psi|^2 of what it stores
//            (FP64 across chunks of 16 points) and its last block turns the
//            per-tile partials, in a fixed order, into the factor 1 / sqrt(norm)
//            that the next x sweep applies.
//
// Thomas recurrence with precomputed elimination coefficients for the system
// (1+2a) u_j - a (u_{j-1} + u_{j+1}) = (1-2a) v_j + a (v_{j-1} + v_{j+1}):
//   forward   d_j = A_j v_j + B_j (v_{j-1} + v_{j+1} + d_{j-1}),
//   back      u_j = d_j + B_j u_{j+1},
// with A_j = m_j (1 - 2a), B_j = a m_j and m_j the pivots (computed in FP64 on
// the host).  The forward values overwrite the tile in place; the three values
// v_{j-1}, v_j, v_{j+1} the right-hand side needs ride in registers.
#include "gp_device.cuh"

namespace gpk {

// ----------------------------------------------------------- field policies

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
  static __device__ __forceinline__ E forward(E A, E B, E prev, E next, E dprev, E cur) {
    return fma(B, prev + next + dprev, A * cur);
  }
  static __device__ __forceinline__ E back(E B, E unext, E d) { return fma(B, unext, d); }
  static __device__ __forceinline__ R abs2(E v) { return v * v; }
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
  static __device__ __forceinline__ E forward(E A, E B, E prev, E next, E dprev, E cur) {
    return cfma(B, cadd(cadd(prev, next), dprev), cmul(A, cur));
  }
  static __device__ __forceinline__ E back(E B, E unext, E d) { return cfma(B, unext, d); }
  static __device__ __forceinline__ R abs2(E v) { return fma(v.x, v.x, v.y * v.y); }
};

// ------------------------------------------------------------------ sweep x

template <class R, bool CPLX>
__global__ void __launch_bounds__(32) k_sweep_x(const SweepParams p) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x;
  const int P = p.pitch, nx = p.nx, W = p.lines;
  const long long nrows = (long long)p.ny * p.nz;
  const long long r0 = (long long)blockIdx.x * W;
  const int rows = (int)min((long long)W, nrows - r0);
  E* tile = reinterpret_cast<E*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)W * P * sizeof(E));
  E* gtile = reinterpret_cast<E*>(p.psi) + r0 * P;
  const uint32_t bytes = (uint32_t)((size_t)rows * P * sizeof(E));

  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, bytes);
    bulk_load(tile, gtile, bytes, bar);
  }
  __syncwarp();
  if (!wait_tile(bar, p.status)) return;

  if (lane < rows) {
    const long long r = r0 + lane;
    const int j = (int)(r % p.ny);
    const int k = (int)(r / p.ny);
    const R* vx = static_cast<const R*>(p.vx);
    const R vyz = __ldg(static_cast<const R*>(p.vy) + j) + __ldg(static_cast<const R*>(p.vz) + k);
    const R s = (R)(*p.scale);
    const R dt = (R)p.dt, g = (R)p.g;
    const E* A = static_cast<const E*>(p.A);
    const E* B = static_cast<const E*>(p.B);
    E* row = tile + (size_t)lane * P;
    const int sig = (P & 1) ? 0 : 1;  // skew the wavefront when the pitch is even
    const int span = nx + sig * (W - 1);

    E prev = F::zero(), dprev = F::zero();
    E cur = F::pointwise(F::scaled(row[0], s), __ldg(vx) + vyz, dt, g);
    for (int t = 0; t < span; ++t) {
      const int i = t - sig * lane;
      if (i >= 0 && i < nx) {
        E next = F::zero();
        if (i + 1 < nx) next = F::pointwise(F::scaled(row[i + 1], s), __ldg(vx + i + 1) + vyz, dt, g);
        const E d = F::forward(__ldg(A + i), __ldg(B + i), prev, next, dprev, cur);
        row[i] = d;
        prev = cur;
        cur = next;
        dprev = d;
      }
    }
    E unext = F::zero();
    for (int t = 0; t < span; ++t) {
      const int i = nx - 1 - (t - sig * lane);
      if (i >= 0 && i < nx) {
        const E u = F::back(__ldg(B + i), unext, row[i]);
        row[i] = u;
        unext = u;
      }
    }
  }
  fence_smem_to_async();
  __syncwarp();
  if (lane == 0) {
    bulk_store(gtile, tile, bytes);
    bulk_commit();
    bulk_wait_read_all();
  }
}

// -------------------------------------------------------- column Thomas solve

// Solve the W columns of a [n][W] tile in place; lane l owns column l.  With NORM
// the sum of |u|^2 over the column is returned (FP32 chunks of 16 folded into FP64).
template <class R, bool CPLX, bool NORM>
__device__ __forceinline__ double solve_columns(typename Field<R, CPLX>::E* tile, int W, int n,
                                                const typename Field<R, CPLX>::E* A,
                                                const typename Field<R, CPLX>::E* B) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  const int lane = threadIdx.x;
  double acc = 0.0;
  if (lane >= W) return acc;
  E* col = tile + lane;
  E prev = F::zero(), dprev = F::zero(), cur = col[0];
  for (int j = 0; j < n; ++j) {
    const E next = (j + 1 < n) ? col[(size_t)(j + 1) * W] : F::zero();
    const E d = F::forward(__ldg(A + j), __ldg(B + j), prev, next, dprev, cur);
    col[(size_t)j * W] = d;
    prev = cur;
    cur = next;
    dprev = d;
  }
  E unext = F::zero();
  R part = R(0);
  int cnt = 0;
  for (int j = n - 1; j >= 0; --j) {
    const E u = F::back(__ldg(B + j), unext, col[(size_t)j * W]);
    col[(size_t)j * W] = u;
    unext = u;
    if (NORM) {
      part += F::abs2(u);
      if (++cnt == 16) {
        acc += (double)part;
        part = R(0);
        cnt = 0;
      }
    }
  }
  if (NORM) acc += (double)part;
  return acc;
}

// ------------------------------------------------------------------ sweep y

template <class R, bool CPLX>
__global__ void __launch_bounds__(32) k_sweep_y(const __grid_constant__ CUtensorMap map,
                                                const SweepParams p) {
  using E = typename Field<R, CPLX>::E;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x;
  const int W = p.lines;
  const int i0 = blockIdx.x * W;
  const int k = blockIdx.y;
  E* tile = reinterpret_cast<E*>(smem);
  const size_t box_bytes = (size_t)p.box * W * sizeof(E);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + box_bytes * p.nbox);
  const int cx = i0 * p.words_per_elem;

  if (lane == 0) {
    prefetch_tmap(&map);
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, (uint32_t)(box_bytes * p.nbox));
    for (int c = 0; c < p.nbox; ++c)
      tma_load_3d(smem + c * box_bytes, &map, cx, c * p.box, k, bar);
  }
  __syncwarp();
  if (!wait_tile(bar, p.status)) return;
  solve_columns<R, CPLX, false>(tile, W, p.n, static_cast<const E*>(p.A),
                                static_cast<const E*>(p.B));
  fence_smem_to_async();
  __syncwarp();
  if (lane == 0) {
    for (int c = 0; c < p.nbox; ++c) tma_store_3d(&map, cx, c * p.box, k, smem + c * box_bytes);
    bulk_commit();
    bulk_wait_read_all();
  }
}

// ------------------------------------------------------------------ sweep z

template <class R, bool CPLX, bool NORM>
__global__ void __launch_bounds__(32) k_sweep_z(const __grid_constant__ CUtensorMap map,
                                                const SweepParams p) {
  using E = typename Field<R, CPLX>::E;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x;
  const int W = p.lines;
  const int i0 = blockIdx.x * W;
  const int j = blockIdx.y;
  E* tile = reinterpret_cast<E*>(smem);
  const size_t box_bytes = (size_t)p.box * W * sizeof(E);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + box_bytes * p.nbox);
  const int cx = i0 * p.words_per_elem;

  if (lane == 0) {
    prefetch_tmap(&map);
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, (uint32_t)(box_bytes * p.nbox));
    for (int c = 0; c < p.nbox; ++c)
      tma_load_3d(smem + c * box_bytes, &map, cx, j, c * p.box, bar);
  }
  __syncwarp();
  double acc = 0.0;
  if (wait_tile(bar, p.status)) {
    acc = solve_columns<R, CPLX, NORM>(tile, W, p.n, static_cast<const E*>(p.A),
                                       static_cast<const E*>(p.B));
    fence_smem_to_async();
    __syncwarp();
    if (lane == 0) {
      for (int c = 0; c < p.nbox; ++c) tma_store_3d(&map, cx, j, c * p.box, smem + c * box_bytes);
      bulk_commit();
      bulk_wait_read_all();
    }
  }
  if constexpr (NORM) {
  // Fixed-order warp sum, per-tile partial, and the last block's final sum.
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  int last = 0;
  if (lane == 0) {
    const long long tile_id = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    p.partials[tile_id] = acc;
    __threadfence();
    const unsigned int ticket = atomicAdd(p.counter, 1u);
    last = (ticket == (unsigned int)(p.ntiles - 1));
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
  __threadfence();
  double s = 0.0, c = 0.0;  // Neumaier
  for (long long t = lane; t < p.ntiles; t += 32) {
    const double x = __ldcg(p.partials + t);
    const double u = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - u) + x : (x - u) + s;
    s = u;
  }
  s += c;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double norm = s * p.dV;
    if (!(norm > 0.0) || !isfinite(norm)) atomicOr(p.status, kStatusNonFinite);
    *p.scale_out = 1.0 / sqrt(norm);
    *p.counter = 0u;
  }
  }
  }
}

// ---------------------------------------------------------------- launchers

template <class R>
cudaError_t launch_sweep_x(const SweepParams& p, bool complex_field, size_t smem,
                           cudaStream_t st) {
  const long long nrows = (long long)p.ny * p.nz;
  const dim3 grid((unsigned int)((nrows + p.lines - 1) / p.lines));
  if (complex_field)
    k_sweep_x<R, true><<<grid, 32, smem, st>>>(p);
  else
    k_sweep_x<R, false><<<grid, 32, smem, st>>>(p);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_sweep_y(const CUtensorMap& map, const SweepParams& p, bool complex_field,
                           size_t smem, cudaStream_t st) {
  const dim3 grid((unsigned int)p.tiles_x, (unsigned int)p.nz);
  if (complex_field)
    k_sweep_y<R, true><<<grid, 32, smem, st>>>(map, p);
  else
    k_sweep_y<R, false><<<grid, 32, smem, st>>>(map, p);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_sweep_z(const CUtensorMap& map, const SweepParams& p, bool complex_field,
                           size_t smem, cudaStream_t st) {
  const dim3 grid((unsigned int)p.tiles_x, (unsigned int)p.ny);
  if (complex_field)
    k_sweep_z<R, true, false><<<grid, 32, smem, st>>>(map, p);
  else
    k_sweep_z<R, false, true><<<grid, 32, smem, st>>>(map, p);
  return cudaGetLastError();
}

template <class R> cudaError_t sweep_set_smem_limits(size_t max_smem) {
  const int b = (int)max_smem;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_sweep_x<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep_x<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep_y<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep_y<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep_z<R, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep_z<R, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  return cudaSuccess;
}

template cudaError_t launch_sweep_x<double>(const SweepParams&, bool, size_t, cudaStream_t);
template cudaError_t launch_sweep_x<float>(const SweepParams&, bool, size_t, cudaStream_t);
template cudaError_t launch_sweep_y<double>(const CUtensorMap&, const SweepParams&, bool, size_t, cudaStream_t);
template cudaError_t launch_sweep_y<float>(const CUtensorMap&, const SweepParams&, bool, size_t, cudaStream_t);
template cudaError_t launch_sweep_z<double>(const CUtensorMap&, const SweepParams&, bool, size_t, cudaStream_t);
template cudaError_t launch_sweep_z<float>(const CUtensorMap&, const SweepParams&, bool, size_t, cudaStream_t);
template cudaError_t sweep_set_smem_limits<double>(size_t);
template cudaError_t sweep_set_smem_limits<float>(size_t);

}  // namespace gpk
