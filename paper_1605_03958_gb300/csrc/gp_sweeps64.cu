// gp_sweeps64.cu -- the Crank-Nicolson sweeps of one split-step Crank-Nicolson step for
// fields stored in FP64 (the paper's precision): the real field of imaginary time and
// the complex field of real time (paper, program summary: "Solution method"; imag3d /
// real3d summaries).  Same method and recurrence as the tile kernels of gp_sweeps.cu:
//   forward   d_j = B_j d_{j-1} + [A_j v_j + B_j (v_{j-1} + v_{j+1})],
//   back      u_j = d_j + B_j u_{j+1},
// A_j = m_j (1 - 2a), B_j = a m_j, m_j the Thomas pivots (computed in FP64 on the host).
//
// FP64 arithmetic is narrow on this part: the whole GPU retires about 0.5 T FP64 lane
// operations per second (FP32: 35 T), a warp's FP64 instruction costs the same with
// any number of active lanes, and one warp per scheduler keeps a scheduler's FP64 unit
// busy (a dependent FP64 chain hides its latency at that rate).  So these kernels
//   * keep all 32 lanes of every warp on useful work,
//   * spread their warps evenly over the SMs' schedulers (no full-line shared-memory
//     tile: occupancy is set by registers, not by the line length),
//   * spend as few FP64 instructions per point as the method allows: 13 for x with the
//     pointwise substep (real field; the exp polynomial's degree chosen per group of
//     points from a bound on its argument), 5 for y and z, 1 more in z for the norm.
// Memory traffic is secondary: a sweep reads and writes the field twice (forward values
// stored in place, then the back substitution), mostly through L2, in a fraction of
// its arithmetic time.
//
//   x    a warp owns 32 consecutive rows, one row per lane.  Rows are contiguous, so a
//        warp moves them through shared memory in chunks of C columns (32 real / 16
//        complex, padded rows against bank conflicts): a chunk is loaded and stored
//        coalesced (lane = column) and the recurrence walks it lane = row.  The pending
//        renormalisation factor and the pointwise substep are applied on the load.
//   y/z  a thread owns one line; lanes are consecutive x, so every access is coalesced.
//        The line streams forward (forward values in place) and back, loads issued kU
//        elements ahead.  z sums |u|^2 of its output for the renormalisation factor.
#include "gp_device.cuh"

namespace gpk {

namespace {

constexpr int kU64 = 8;          // y / z: elements loaded ahead of the recurrence
constexpr int kX64Warps = 4;     // x: warps per block (each on its own 32 rows)
constexpr int kLineThreads = 128;

// (-1)^k / k!, k = 0..9: the Taylor coefficients of exp(-y)
__device__ constexpr double kSignedInvFact[10] = {
    1.0, -1.0, 1.0 / 2.0, -1.0 / 6.0, 1.0 / 24.0, -1.0 / 120.0, 1.0 / 720.0, -1.0 / 5040.0,
    1.0 / 40320.0, -1.0 / 362880.0};

template <class E>
__device__ __forceinline__ E coef64(const E* T, int j, int head, E bulk) {
  return j < head ? __ldg(T + j) : bulk;
}

// |y| as an ordered integer (IEEE-754 bits without the sign); NaN sorts above every
// finite bound, so a NaN takes the library branch and propagates.
__device__ __forceinline__ unsigned long long abs_bits(double y) {
  return (unsigned long long)__double_as_longlong(y) & 0x7fffffffffffffffull;
}
// Bounds on the argument of exp(-y) / cis(-y) for the Taylor polynomials below: their
// remainders stay under 2^-56 (a quarter of an FP64 ulp of 1).
constexpr unsigned long long kBits2m10 = 0x3F50000000000000ull;  // 2^-10: exp, degree 4
constexpr unsigned long long kBits2m8 = 0x3F70000000000000ull;   // 2^-8:  cos 4 / sin 5
constexpr unsigned long long kBits2m7 = 0x3F80000000000000ull;   // 2^-7:  exp, degree 6
constexpr unsigned long long kBits2m4 = 0x3FB0000000000000ull;   // 2^-4:  exp 9, cos 8 / sin 9

// Pointwise substep of one chunk group on load (lane = column).  x[u] are raw field
// values of NG rows of one column; rf[u] their rows' trap factors exp(-dt (V_y + V_z))
// (or cis(-dt (V_y + V_z))); the column's factor exp(-dt V_x) and the pending scale s
// are folded into the polynomial's coefficients c[k] = s fx (-1)^k / k!.
//   real:    v <- (x rf) * sum_k c_k y^k,   y = (dt g s^2) x^2
//            -- 8 FP64 instructions per point at degree 4 (x^2, y, x rf, 4 Horner, 1)
template <int NG>
__device__ __forceinline__ void pointwise_real(double (&x)[NG], const double (&rf)[NG],
                                               const double (&c)[10], double cy) {
  double y[NG];
  unsigned long long mb = 0;
#pragma unroll
  for (int u = 0; u < NG; ++u) {
    y[u] = cy * (x[u] * x[u]);
    mb = max(mb, abs_bits(y[u]));
    x[u] = x[u] * rf[u];
  }
  if (__all_sync(0xffffffffu, mb <= kBits2m10)) {
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      double q = fma(y[u], c[4], c[3]);
      q = fma(y[u], q, c[2]);
      q = fma(y[u], q, c[1]);
      x[u] *= fma(y[u], q, c[0]);
    }
  } else if (__all_sync(0xffffffffu, mb <= kBits2m7)) {
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      double q = fma(y[u], c[6], c[5]);
#pragma unroll
      for (int k = 4; k >= 1; --k) q = fma(y[u], q, c[k]);
      x[u] *= fma(y[u], q, c[0]);
    }
  } else if (__all_sync(0xffffffffu, mb <= kBits2m4)) {
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      double q = fma(y[u], c[9], c[8]);
#pragma unroll
      for (int k = 7; k >= 1; --k) q = fma(y[u], q, c[k]);
      x[u] *= fma(y[u], q, c[0]);
    }
  } else {
#pragma unroll
    for (int u = 0; u < NG; ++u) x[u] *= c[0] * exp(-y[u]);
  }
}

//   complex: v <- (x rf) * (G (cos th - i sin th)),  th = (dt g s^2) |x|^2, G = s fx
//            -- 21 FP64 instructions per point with the degree-4 / 5 polynomials
template <int NG>
__device__ __forceinline__ void pointwise_cplx(double2 (&x)[NG], const double2 (&rf)[NG],
                                               double2 G, double cy) {
  double th[NG];
  unsigned long long mb = 0;
#pragma unroll
  for (int u = 0; u < NG; ++u) {
    th[u] = cy * fma(x[u].x, x[u].x, x[u].y * x[u].y);
    mb = max(mb, abs_bits(th[u]));
    x[u] = cmul(x[u], rf[u]);
  }
  double cs[NG], sn[NG];
  if (__all_sync(0xffffffffu, mb <= kBits2m8)) {
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      const double t2 = th[u] * th[u];
      cs[u] = fma(t2, fma(t2, 1.0 / 24.0, -0.5), 1.0);
      sn[u] = th[u] * fma(t2, fma(t2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    }
  } else if (__all_sync(0xffffffffu, mb <= kBits2m4)) {
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      const double t2 = th[u] * th[u];
      double c = fma(t2, 1.0 / 40320.0, -1.0 / 720.0);
      c = fma(t2, c, 1.0 / 24.0);
      c = fma(t2, c, -0.5);
      cs[u] = fma(t2, c, 1.0);
      double s = fma(t2, 1.0 / 362880.0, -1.0 / 5040.0);
      s = fma(t2, s, 1.0 / 120.0);
      s = fma(t2, s, -1.0 / 6.0);
      sn[u] = th[u] * fma(t2, s, 1.0);
    }
  } else {
#pragma unroll
    for (int u = 0; u < NG; ++u) sincos(th[u], &sn[u], &cs[u]);
  }
#pragma unroll
  for (int u = 0; u < NG; ++u) {
    // H = G (cs - i sn)
    const double2 H = make_double2(fma(G.x, cs[u], G.y * sn[u]), fma(G.y, cs[u], -G.x * sn[u]));
    x[u] = cmul(x[u], H);
  }
}

}  // namespace

// ------------------------------------------------------------------ sweep x

template <bool CPLX> struct X64Geom {
  using E = typename Field<double, CPLX>::E;
  static constexpr int C = CPLX ? 16 : 32;   // columns per chunk
  static constexpr int LD = C + 1;           // padded chunk row, elements
  static constexpr int RPI = 32 / C;         // rows per 32-lane load
  static constexpr int NG = 8;               // loads in flight per lane
  static constexpr size_t warp_elems = 2 * 32 * LD + 32;   // two chunk buffers + row factors
  static constexpr size_t smem = kX64Warps * warp_elems * sizeof(E);
};

template <bool CPLX>
__global__ void __launch_bounds__(kX64Warps * 32) k_sweep_x64(const __grid_constant__ SweepParams p) {
  using F = Field<double, CPLX>;
  using E = typename F::E;
  using G = X64Geom<CPLX>;
  constexpr int C = G::C, LD = G::LD, RPI = G::RPI, NG = G::NG;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  E* wbase = reinterpret_cast<E*>(smem) + (size_t)wib * G::warp_elems;
  auto buf = [&](int c) { return wbase + (c & 1) * (32 * LD); };   // chunk c's buffer
  E* rowf = wbase + 2 * 32 * LD;
  const long long nrows = (long long)p.ny * p.nz;
  const long long r0 = ((long long)blockIdx.x * kX64Warps + wib) * 32;
  pdl_begin();
  if (r0 >= nrows) return;
  const int rows = (int)min(32LL, nrows - r0);
  const int nx = p.nx, P = p.pitch, head = p.head;
  E* field = static_cast<E*>(p.psi) + (size_t)r0 * P;
  const double s = *p.scale;
  const bool pw = p.pw != 0;
  const double cy = p.dt * p.g * s * s;
  const E* fx = static_cast<const E*>(p.band_fx);
  const E* A = static_cast<const E*>(p.A);
  const E* B = static_cast<const E*>(p.B);
  const E Ab = __ldg(A + nx - 1), Bb = __ldg(B + nx - 1);
  rowf[lane] = lane < rows ? __ldg(static_cast<const E*>(p.band_fyz) + r0 + lane) : F::zero();
  __syncwarp();

  const int lc = lane % C, lr = lane / C;   // load geometry: column and row offset
  const int nch = (nx + C - 1) / C;

  // chunk c of the warp's rows into b, lane = column: pending factor and pointwise
  // substep applied (columns past nx and rows past `rows` read as zero)
  auto load_chunk = [&](int c, E* b) {
    const int col = c * C + lc;
    const bool cin = col < nx;
    const E f = cin ? __ldg(fx + col) : F::zero();
    double cr[10];
    double2 Gc = make_double2(0.0, 0.0);
    if constexpr (!CPLX) {
      const double sf = s * f;
#pragma unroll
      for (int k = 0; k < 10; ++k) cr[k] = sf * kSignedInvFact[k];   // s fx (-1)^k / k!
    } else {
      Gc = make_double2(s * f.x, s * f.y);
    }
#pragma unroll
    for (int g0 = 0; g0 < 32; g0 += NG * RPI) {
      E xv[NG], rf[NG];
#pragma unroll
      for (int u = 0; u < NG; ++u) {
        const int rho = g0 + u * RPI + lr;
        xv[u] = (cin && rho < rows && GP_IN((r0 + rho) * P + col, nrows * P, p.status))
                    ? field[(size_t)rho * P + col] : F::zero();
        rf[u] = rowf[rho];
      }
      if (!pw) {
#pragma unroll
        for (int u = 0; u < NG; ++u) xv[u] = F::scaled(xv[u], s);
      } else if constexpr (!CPLX) {
        pointwise_real<NG>(xv, rf, cr, cy);
      } else {
        pointwise_cplx<NG>(xv, rf, Gc, cy);
      }
#pragma unroll
      for (int u = 0; u < NG; ++u) b[(g0 + u * RPI + lr) * LD + lc] = xv[u];
    }
  };
  // chunk c of b to the field, lane = column
  auto store_chunk = [&](int c, const E* b) {
    const int col = c * C + lc;
    if (col >= nx) return;
#pragma unroll 8
    for (int rr = 0; rr < 32; rr += RPI) {
      const int rho = rr + lr;
      if (rho < rows && GP_IN((r0 + rho) * P + col, nrows * P, p.status))
        field[(size_t)rho * P + col] = b[rho * LD + lc];
    }
  };
  // forward values of chunk c's v (lane = row), in place; the element after the
  // chunk comes from the next chunk's buffer
  E prev = F::zero(), dprev = F::zero();
  auto forward = [&](int c, E* b, const E* bn) {
    E* rowp = b + lane * LD;
    const int j0 = c * C;
#pragma unroll
    for (int jj = 0; jj < C; ++jj) {
      const int j = j0 + jj;
      if (j < nx) {
        const E cur = rowp[jj];
        const E nxt = jj + 1 < C ? rowp[jj + 1] : (j + 1 < nx ? bn[lane * LD] : F::zero());
        const E bj = coef64(B, j, head, Bb);
        const E d = F::chain(bj, dprev, F::rhs(coef64(A, j, head, Ab), bj, prev, nxt, cur));
        rowp[jj] = d;
        prev = cur;
        dprev = d;
      }
    }
  };
  E unext = F::zero();
  auto back = [&](int c, E* b) {
    E* rowp = b + lane * LD;
    const int j0 = c * C;
#pragma unroll
    for (int jj = C - 1; jj >= 0; --jj) {
      const int j = j0 + jj;
      if (j < nx) {
        const E u = F::chain(coef64(B, j, head, Bb), unext, rowp[jj]);
        rowp[jj] = u;
        unext = u;
      }
    }
  };

  load_chunk(0, buf(0));
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) load_chunk(c + 1, buf(c + 1));
    __syncwarp();
    forward(c, buf(c), buf(c + 1));
    __syncwarp();
    // the last chunk's forward values stay in shared memory for the back substitution
    if (c + 1 < nch) store_chunk(c, buf(c));
  }
  for (int c = nch - 1; c >= 0; --c) {
    E* b = buf(c);
    if (c + 1 < nch) {
      const int col = c * C + lc;   // plain copy of the forward values back in
#pragma unroll 8
      for (int rr = 0; rr < 32; rr += RPI) {
        const int rho = rr + lr;
        b[rho * LD + lc] = (col < nx && rho < rows && GP_IN((r0 + rho) * P + col, nrows * P, p.status))
                               ? field[(size_t)rho * P + col] : F::zero();
      }
      __syncwarp();
    }
    back(c, b);
    __syncwarp();
    store_chunk(c, b);
  }
}

// -------------------------------------------------------------- sweeps y, z

// AXIS 1 (y) or 2 (z): thread g owns line (i = g mod nx, c = g / nx), c the z index
// (y sweep) or the y index (z sweep).  With NORM the block sums |u|^2 and the last
// block turns the partials into the renormalisation factor.
template <bool CPLX, int AXIS, bool NORM>
__global__ void __launch_bounds__(kLineThreads) k_sweep_line64(const __grid_constant__ SweepParams p) {
  using F = Field<double, CPLX>;
  using E = typename F::E;
  pdl_begin();
  const int nx = p.nx, n = p.n, head = p.head;
  const long long nlines = (long long)nx * (AXIS == 1 ? p.nz : p.ny);
  const long long g = (long long)blockIdx.x * kLineThreads + threadIdx.x;
  double acc = 0.0;
  const int i = (int)(g % nx);
  const long long c = g / nx;
  const size_t P = (size_t)p.pitch;
  const size_t stride = AXIS == 1 ? P : P * (size_t)p.ny;
  const size_t first = (AXIS == 1 ? (size_t)c * P * p.ny : (size_t)c * P) + i;
  // the line's last element inside the field (bounds checks; the block still reaches
  // the norm's barriers)
  if (g < nlines && GP_IN(first + (size_t)(n - 1) * stride, (long long)p.nz * p.ny * (long long)P, p.status)) {
    E* line = static_cast<E*>(p.psi) + first;
    const E* A = static_cast<const E*>(p.A);
    const E* B = static_cast<const E*>(p.B);
    const E Ab = __ldg(A + n - 1), Bb = __ldg(B + n - 1);
    auto rd = [&](int j) -> E { return (j >= 0 && j < n) ? line[(size_t)j * stride] : F::zero(); };

    E prev = F::zero(), dprev = F::zero(), cur = rd(0);
    E nxt[kU64];
#pragma unroll
    for (int u = 0; u < kU64; ++u) nxt[u] = rd(u + 1);
    for (int j0 = 0; j0 < n; j0 += kU64) {
      E pre[kU64];
#pragma unroll
      for (int u = 0; u < kU64; ++u) pre[u] = rd(j0 + kU64 + u + 1);
#pragma unroll
      for (int u = 0; u < kU64; ++u) {
        const int j = j0 + u;
        if (j < n) {
          const E b = coef64(B, j, head, Bb);
          const E d = F::chain(b, dprev, F::rhs(coef64(A, j, head, Ab), b, prev, nxt[u], cur));
          line[(size_t)j * stride] = d;
          prev = cur;
          cur = nxt[u];
          dprev = d;
        }
      }
#pragma unroll
      for (int u = 0; u < kU64; ++u) nxt[u] = pre[u];
    }

    E unext = F::zero();
    E dv[kU64];
#pragma unroll
    for (int u = 0; u < kU64; ++u) dv[u] = rd(n - 1 - u);
    for (int j0 = n - 1; j0 >= 0; j0 -= kU64) {
      E pre[kU64];
#pragma unroll
      for (int u = 0; u < kU64; ++u) pre[u] = rd(j0 - kU64 - u);
#pragma unroll
      for (int u = 0; u < kU64; ++u) {
        const int j = j0 - u;
        if (j >= 0) {
          const E v = F::chain(coef64(B, j, head, Bb), unext, dv[u]);
          line[(size_t)j * stride] = v;
          unext = v;
          if constexpr (NORM) acc = fma(v, v, acc);
        }
      }
#pragma unroll
      for (int u = 0; u < kU64; ++u) dv[u] = pre[u];
    }
  }
  if constexpr (NORM) norm_finish(acc, p.partials, p.counter, gridDim.x, blockIdx.x, p.scale_out,
                                  p.status, p.dV);
}

// ------------------------------------------------------------------ launchers

size_t x64_smem(bool complex_field) {
  return complex_field ? X64Geom<true>::smem : X64Geom<false>::smem;
}

cudaError_t sweep64_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_sweep_x64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)X64Geom<false>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sweep_x64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)X64Geom<true>::smem);
  return e;
}

long long sweep64_blocks(int axis, int nx, int ny, int nz) {
  if (axis == 0) {
    const long long warps = ((long long)ny * nz + 31) / 32;
    return (warps + kX64Warps - 1) / kX64Warps;
  }
  const long long lines = (long long)nx * (axis == 1 ? nz : ny);
  return (lines + kLineThreads - 1) / kLineThreads;
}

cudaError_t launch_sweep64(int axis, const SweepParams& p, bool complex_field, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.stream = st;
  cfg.gridDim = dim3((unsigned)sweep64_blocks(axis, p.nx, p.ny, p.nz));
  if (axis == 0) {
    cfg.blockDim = dim3(kX64Warps * 32);
    cfg.dynamicSmemBytes = x64_smem(complex_field);
    return complex_field ? cudaLaunchKernelEx(&cfg, k_sweep_x64<true>, p)
                         : cudaLaunchKernelEx(&cfg, k_sweep_x64<false>, p);
  }
  cfg.blockDim = dim3(kLineThreads);
  if (axis == 1)
    return complex_field ? cudaLaunchKernelEx(&cfg, k_sweep_line64<true, 1, false>, p)
                         : cudaLaunchKernelEx(&cfg, k_sweep_line64<false, 1, false>, p);
  // the norm is summed in imaginary time only (real field)
  return complex_field ? cudaLaunchKernelEx(&cfg, k_sweep_line64<true, 2, false>, p)
                       : cudaLaunchKernelEx(&cfg, k_sweep_line64<false, 2, true>, p);
}

}  // namespace gpk
