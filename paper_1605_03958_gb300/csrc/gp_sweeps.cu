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
//   forward   d_j = B_j d_{j-1} + [A_j v_j + B_j (v_{j-1} + v_{j+1})],
//   back      u_j = d_j + B_j u_{j+1},
// with A_j = m_j (1 - 2a), B_j = a m_j and m_j the pivots (computed in FP64 on
// the host).  Only the first FMA of each line is on the recurrence's dependency
// chain; the bracket is computed off it.  The forward values overwrite the tile in
// place; the neighbours v_{j-1}, v_j, v_{j+1} ride in registers and the next kU
// tile values are loaded a chunk ahead, so shared-memory latency is off the chain.
// The pivots converge geometrically; from index `head` on, the coefficients rounded
// to the storage precision are all equal to the last one (the host checks this
// exactly), so the bulk of a line takes them from registers and only the first
// `head` entries come from the table.
#include <algorithm>

#include <utility>

#include "gp_device.cuh"

namespace gpk {

constexpr int kU = 8;  // elements loaded ahead of the recurrence

template <class E>
__device__ __forceinline__ E coef(const E* T, int j, int head, E bulk) {
  return j < head ? __ldg(T + j) : bulk;
}

// ------------------------------------------------------------------ sweep x

template <class R, bool CPLX>
__global__ void __launch_bounds__(32) k_sweep_x(const SweepParams p) {
  pdl_begin();
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
  if (!GP_IN((r0 + rows) * P - 1, nrows * P, p.status)) return;

  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, bytes);
    bulk_load(tile, gtile, bytes, bar);
  }
  __syncwarp();
  if (!wait_tile(bar, p.status, p.wait_ns)) return;

  if (lane < rows) {
    const long long r = r0 + lane;
    const int j = (int)(r % p.ny);
    const int k = (int)(r / p.ny);
    const E* fxt = static_cast<const E*>(p.band_fx);                      // trap factor along x
    const E fr = __ldg(static_cast<const E*>(p.band_fyz) + (size_t)k * p.ny + j);   // of this row
    const R s = (R)(*p.scale) * (R)step_dither_f(p.step_ctr);
    const R dtg = (R)(p.dt * p.g);
    const E* A = static_cast<const E*>(p.A);
    const E* B = static_cast<const E*>(p.B);
    const int head = p.head;
    const E Ab = __ldg(A + nx - 1), Bb = __ldg(B + nx - 1);
    E* row = tile + (size_t)lane * P;
    // Lane l walks its row delayed by `off` steps: at step t it handles element
    // t - off.  With an even pitch the 32 lanes then touch 32 different banks.
    const int sig = (P & 1) ? 0 : 1;
    const int off = sig * lane;
    const int span = nx + sig * (W - 1);
    // element idx after the pending scale and the pointwise substep (0 outside)
    auto load = [&](int idx) -> E {
      if (idx < 0 || idx >= nx) return F::zero();
      const E v = F::scaled(row[idx], s);
      if (!p.pw) return v;   // kinetic-only step
      const R y = dtg * F::abs2(v);
      const E f = F::mul(__ldg(fxt + idx), fr);
      return fabs(y) <= R(0.0625) ? F::nonlinear_small(v, f, y) : F::nonlinear_full(v, f, y);
    };

    E prev = F::zero(), dprev = F::zero();
    E cur = load(0);
    E nxt[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) nxt[u] = load(u + 1 - off);
    for (int tc = 0; tc < span; tc += kU) {
      E pre[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) pre[u] = load(tc + kU + u + 1 - off);
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = tc + u - off;
        if (i >= 0 && i < nx) {
          const E b = coef(B, i, head, Bb);
          const E d = F::chain(b, dprev, F::rhs(coef(A, i, head, Ab), b, prev, nxt[u], cur));
          row[i] = d;
          prev = cur;
          cur = nxt[u];
          dprev = d;
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) nxt[u] = pre[u];
    }
    // back substitution, element nx-1-(t-off) at step t
    auto rd = [&](int idx) -> E { return (idx >= 0 && idx < nx) ? row[idx] : F::zero(); };
    E unext = F::zero();
    E dv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) dv[u] = rd(nx - 1 + off - u);
    for (int tc = 0; tc < span; tc += kU) {
      E pre[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) pre[u] = rd(nx - 1 + off - tc - kU - u);
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = nx - 1 + off - tc - u;
        if (i >= 0 && i < nx) {
          const E v = F::chain(coef(B, i, head, Bb), unext, dv[u]);
          row[i] = v;
          unext = v;
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) dv[u] = pre[u];
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
                                                const typename Field<R, CPLX>::E* B,
                                                int head) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  const int lane = threadIdx.x;
  double acc = 0.0;
  if (lane >= W) return acc;
  E* col = tile + lane;
  const E Ab = __ldg(A + n - 1), Bb = __ldg(B + n - 1);
  auto rd = [&](int j) -> E { return (j >= 0 && j < n) ? col[(size_t)j * W] : F::zero(); };

  E prev = F::zero(), dprev = F::zero(), cur = col[0];
  E nxt[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) nxt[u] = rd(u + 1);
  for (int j0 = 0; j0 < n; j0 += kU) {
    E pre[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) pre[u] = rd(j0 + kU + u + 1);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 + u;
      if (j < n) {
        const E b = coef(B, j, head, Bb);
        const E d = F::chain(b, dprev, F::rhs(coef(A, j, head, Ab), b, prev, nxt[u], cur));
        col[(size_t)j * W] = d;
        prev = cur;
        cur = nxt[u];
        dprev = d;
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) nxt[u] = pre[u];
  }

  E unext = F::zero();
  R part = R(0);
  E dv[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) dv[u] = rd(n - 1 - u);
  for (int j0 = n - 1; j0 >= 0; j0 -= kU) {
    E pre[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) pre[u] = rd(j0 - kU - u);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = j0 - u;
      if (j >= 0) {
        const E v = F::chain(coef(B, j, head, Bb), unext, dv[u]);
        col[(size_t)j * W] = v;
        unext = v;
        if (NORM) part += F::abs2(v);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) dv[u] = pre[u];
    if (NORM && ((n - 1 - j0) / kU) % 2 == 1) {  // fold into FP64 every 16 elements
      acc += (double)part;
      part = R(0);
    }
  }
  if (NORM) acc += (double)part;
  return acc;
}

// ------------------------------------------------------------------ sweep y

template <class R, bool CPLX>
__global__ void __launch_bounds__(32) k_sweep_y(const __grid_constant__ CUtensorMap map,
                                                const SweepParams p) {
  pdl_begin();
  // the factor's dither (FP32, imaginary time): the step's x sweep has read the counter
  if (p.step_ctr && blockIdx.x == 0 && threadIdx.x == 0) *p.step_ctr += 1;
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
  if (!wait_tile(bar, p.status, p.wait_ns)) return;
  solve_columns<R, CPLX, false>(tile, W, p.n, static_cast<const E*>(p.A),
                                static_cast<const E*>(p.B), p.head);
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
  pdl_begin();
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
  if (wait_tile(bar, p.status, p.wait_ns)) {
    acc = solve_columns<R, CPLX, NORM>(tile, W, p.n, static_cast<const E*>(p.A),
                                       static_cast<const E*>(p.B), p.head);
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

// ============================================================================
// Shared-memory-free FP32 sweeps (real and complex fields).
//
// In the bulk of a line every rounded coefficient equals (A, B) (see `head`), and
// |B| < 1, so the coupling between elements decays like |B|^distance.  The host
// picks a truncation depth L with |B|^(L+1) <= 2^-30 (below an FP32 ulp); both
// kernels below cut the coupling there and are otherwise the same recurrence:
//  * back substitution u_e = d_e + B u_{e+1} in the bulk equals the series
//    sum_{m>=0} B^m d_{e+m}; cut after m = L it becomes a Horner sum over the
//    last L+1 forward values, so a line streams in one direction: u_e is
//    emitted L elements behind the forward recurrence.  At the line end the
//    series ends on its own (d = 0 past the last element: the exact boundary);
//    the first `head` elements, whose coefficients differ, are finished exactly
//    by the recurrence from u_head.
//  * a segment of a line can be solved by a lane that starts the forward
//    recurrence L+1 elements before the segment (from d = 0) and the back
//    recurrence L elements after it (from u = 0).
// ============================================================================

#ifndef GP_STREAM_U
#define GP_STREAM_U 16
#endif
#ifndef GP_STREAM_MINB
#define GP_STREAM_MINB 6
#endif
constexpr int kStreamU = GP_STREAM_U;  // chunk length of the streaming kernel (load lead)
constexpr int kHeadMax = 8;     // largest `head` the streaming kernel handles

__device__ __forceinline__ void norm_block_finish(double acc, const SweepParams& p) {
  norm_finish(acc, p.partials, p.counter, gridDim.x, blockIdx.x, p.scale_out, p.status, p.dV);
}

// y (AXIS 1) or z (AXIS 2) sweep: one lane per line, lanes on consecutive x.  A
// line is split into p.nseg segments handled by different warps; a warp streams
// its segment [s0, s1) with direct coalesced loads, starting the forward
// recurrence L+1 elements early (from d = 0).  The back substitution runs per
// chunk of U elements, L behind the forward: the top element of the chunk is
// seeded by the truncated series sum_{m<=L} B^m d_{e+m}, the rest follow from the
// exact recurrence u_e = d_e + B_e u_{e+1} (table coefficients for e < head).
// The result goes to p.out (not in place: neighbouring segments read each
// other's inputs).
template <class R, bool CPLX, int AXIS, bool NORM, int L>
__global__ void __launch_bounds__(128, CPLX ? 4 : GP_STREAM_MINB) k_sweep_stream(const SweepParams p) {
  pdl_begin();
  // the factor's dither (FP32, imaginary time): the step's x sweep has read the counter
  if (AXIS == 1 && p.step_ctr && blockIdx.x == 0 && threadIdx.x == 0) *p.step_ctr += 1;
  using F = Field<R, CPLX>;
  using E = typename F::E;
  constexpr int U = kStreamU;
  static_assert(L < U && kHeadMax <= U - L, "chunk geometry");
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int tiles_x = p.tiles_x, nseg = p.nseg;
  const int nother = AXIS == 1 ? p.nz : p.ny;
  const bool live = wid < (long long)tiles_x * nother * nseg;
  double acc = 0.0;
  if (live) {
    const int w = (int)wid;
    const int sg = w % nseg;
    const int lw = w / nseg;
    const int tx = lw % tiles_x, o = lw / tiles_x;
    const int i = tx * 32 + lane;
    const bool act = i < p.nx;
    const size_t P = (size_t)p.pitch;
    // lanes past nx mirror column 0 (valid addresses); they store nothing and add
    // nothing to the norm
    const size_t base = (AXIS == 1 ? (size_t)o * p.ny * P : (size_t)o * P) + (act ? i : 0);
    const E* lin = static_cast<const E*>(p.psi) + base;
    E* lout = static_cast<E*>(p.out) + base;
    const size_t st = AXIS == 1 ? P : P * p.ny;
    const int n = p.n, head = p.head;
    const int seglen = (n + nseg - 1) / nseg;
    const int s0 = sg * seglen, s1 = min(n, s0 + seglen);
    const int js = sg == 0 ? 0 : max(0, s0 - L - 1);   // forward start (d = 0 before it)
    const E* A = static_cast<const E*>(p.A);
    const E* B = static_cast<const E*>(p.B);
    const E Ab = __ldg(A + n - 1), Bb = __ldg(B + n - 1);

    E prev = js > 0 ? lin[(size_t)(js - 1) * st] : F::zero();
    E cur = lin[(size_t)js * st];
    E dprev = F::zero();
    E nv[U], tail[L];
    const E* lp = lin + (size_t)(js + 1) * st;   // next element to load
    int jl = js + 1;                              // its index
#pragma unroll
    for (int u = 0; u < U; ++u) {
      nv[u] = jl < n ? *lp : F::zero();
      lp += st;
      ++jl;
    }
#pragma unroll
    for (int q = 0; q < L; ++q) tail[q] = F::zero();
    R part = R(0);
    for (int j0 = js; j0 < s1 + L; j0 += U) {
      E dd[U];
      // forward; each consumed slot of nv is refilled at once with the element U
      // further on, so U loads stay in flight with one register array
      const bool full_load = jl + U <= n;
      if (j0 >= head && j0 + U <= n) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const E nx = nv[u];
          nv[u] = (full_load || jl + u < n) ? *lp : F::zero();
          lp += st;
          const E d = F::chain(Bb, dprev, F::rhs(Ab, Bb, prev, nx, cur));
          prev = cur;
          cur = nx;
          dprev = d;
          dd[u] = d;
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const E nx = nv[u];
          nv[u] = (full_load || jl + u < n) ? *lp : F::zero();
          lp += st;
          const int j = j0 + u;
          if (j < n) {
            const E b = coef(B, j, head, Bb);
            const E d = F::chain(b, dprev, F::rhs(coef(A, j, head, Ab), b, prev, nx, cur));
            prev = cur;
            cur = nx;
            dprev = d;
            dd[u] = d;
          } else {
            dd[u] = F::zero();
          }
        }
      }
      jl += U;
      // back: elements e = j0 - L + u, u = U-1 .. 0; seed at the top
      E un;
      {
        un = dd[U - 1];
#pragma unroll
        for (int m = L - 1; m >= 0; --m) un = F::chain(Bb, un, dd[U - 1 - L + m]);
      }
      const int ebase = j0 - L;
      const bool all_out = ebase >= s0 && ebase + U <= s1 && ebase >= head;
      E* op = lout + (ptrdiff_t)(ebase + U - 1) * (ptrdiff_t)st;
      if (all_out) {
#pragma unroll
        for (int u = U - 1; u >= 0; --u) {
          if (u < U - 1) {  // d_{ebase+u}: dd[u-L] for u >= L, else tail[u]
            const E dv = u >= L ? dd[u >= L ? u - L : 0] : tail[u < L ? u : 0];
            un = F::chain(Bb, un, dv);
          }
          if (act) *op = un;
          op -= st;
          if (NORM && act) part += F::abs2(un);
        }
      } else {
#pragma unroll
        for (int u = U - 1; u >= 0; --u) {
          const int e = ebase + u;
          if (u < U - 1) {
            const E dv = u >= L ? dd[u >= L ? u - L : 0] : tail[u < L ? u : 0];
            const E b = (e >= 0 && e < head) ? __ldg(B + e) : Bb;
            un = F::chain(b, un, dv);
          }
          if (e >= s0 && e < s1 && act) {
            *op = un;
            if (NORM) part += F::abs2(un);
          }
          op -= st;
        }
      }
#pragma unroll
      for (int q = 0; q < L; ++q) tail[q] = dd[U - L + q];
      if (NORM) {
        acc += (double)part;
        part = R(0);
      }
    }
  }
  if (NORM) norm_block_finish(acc, p);
}

// x sweep with the fused pending scale and pointwise substep, streaming form: one
// warp per 32 consecutive rows (lane l owns row r0 + l) in a 32-thread block.  The
// rows advance together in chunks of kXC elements: a chunk of the 32 rows is
// copied with coalesced 4/8-byte cp.async (zero fill past nx) into a padded
// shared-memory tile (stride kXC+1: lane l reading its row touches bank l+u), three
// chunks in flight.  Forward recurrence and the seeded block-backward are those of
// k_sweep_stream; outputs go through a padded tile and leave as coalesced stores.
// Each warp owns whole rows, so the sweep is in place.
constexpr int kXC = 32;            // chunk length along x
constexpr int kXS = kXC + 1;       // padded row stride of a chunk tile

template <class R, bool CPLX, int L>
__global__ void __launch_bounds__(32) k_sweep_x_stream(const SweepParams p) {
  pdl_begin();
  using F = Field<R, CPLX>;
  using E = typename F::E;
  constexpr int C = kXC;
  static_assert(L < C && kHeadMax <= C - L, "chunk geometry");
  extern __shared__ __align__(128) unsigned char smem[];
  E* ib = reinterpret_cast<E*>(smem);          // 3 input tiles [32][kXS]
  E* ob = ib + 3 * 32 * kXS;                    // output tile [32][kXS]
  const int lane = threadIdx.x;
  const long long nrows = (long long)p.ny * p.nz;
  const long long r0 = (long long)blockIdx.x * 32;
  const int rows = (int)min(32LL, nrows - r0);
  const int nx = p.nx, head = p.head;
  const size_t P = (size_t)p.pitch;
  E* field = static_cast<E*>(p.psi) + (size_t)r0 * P;
  const E* A = static_cast<const E*>(p.A);
  const E* B = static_cast<const E*>(p.B);
  const E Ab = __ldg(A + nx - 1), Bb = __ldg(B + nx - 1);
  const R* vx = static_cast<const R*>(p.vx);
  const R s = (R)(*p.scale) * (R)step_dither_f(p.step_ctr);
  const R dt = (R)p.dt, g = (R)p.g;
  const long long myrow = r0 + min(lane, rows - 1);
  const int jrow = (int)(myrow % p.ny), krow = (int)(myrow / p.ny);
  const R vyz = __ldg(static_cast<const R*>(p.vy) + jrow) + __ldg(static_cast<const R*>(p.vz) + krow);
  const int nchunk = (nx + C - 1) / C;

  // chunk c of all 32 rows -> tile c % 3 (always commits a group, maybe empty)
  auto issue = [&](int c) {
    if (c < nchunk) {
      E* t = ib + (c % 3) * 32 * kXS;
      const int j = c * C + lane;
      const bool okj = j < nx;
      for (int q = 0; q < 32; ++q) {
        const bool ok = okj && q < rows;
        const E* src = field + (ok ? (size_t)q * P + j : 0);   // in bounds even when zero-filling
        cp_async_zfill<sizeof(E)>(t + q * kXS + lane, src, ok);
      }
    }
    cp_async_commit();
  };
  // element u of chunk c of this lane's row, after scale and pointwise substep
  auto val = [&](int c, int u) -> E {
    const int j = c * C + u;
    if (j >= nx) return F::zero();
    const E raw = ib[(c % 3) * 32 * kXS + lane * kXS + u];
    if (!p.pw) return F::scaled(raw, s);   // kinetic-only step
    return F::pointwise(F::scaled(raw, s), __ldg(vx + j) + vyz, dt, g);
  };

  issue(0);
  issue(1);
  E prev = F::zero(), dprev = F::zero(), cur = F::zero();
  E tail[L];
#pragma unroll
  for (int q = 0; q < L; ++q) tail[q] = F::zero();
  for (int c = 0; c * C < nx + L; ++c) {
    const int j0 = c * C;
    issue(c + 2);
    cp_async_wait<1>();   // chunks c and c+1 have landed
    __syncwarp();
    if (c == 0) cur = val(0, 0);
    E dd[C];
    if (j0 >= head && j0 + C <= nx) {
#pragma unroll
      for (int u = 0; u < C; ++u) {
        const E nx_ = (u + 1 < C) ? val(c, u + 1) : val(c + 1, 0);
        const E d = F::chain(Bb, dprev, F::rhs(Ab, Bb, prev, nx_, cur));
        prev = cur;
        cur = nx_;
        dprev = d;
        dd[u] = d;
      }
    } else {
#pragma unroll
      for (int u = 0; u < C; ++u) {
        const int j = j0 + u;
        if (j < nx) {
          const E nx_ = (u + 1 < C) ? val(c, u + 1) : val(c + 1, 0);
          const E b = coef(B, j, head, Bb);
          const E d = F::chain(b, dprev, F::rhs(coef(A, j, head, Ab), b, prev, nx_, cur));
          prev = cur;
          cur = nx_;
          dprev = d;
          dd[u] = d;
        } else {
          dd[u] = F::zero();
        }
      }
    }
    // back: e = j0 - L + u, seeded at the top of the chunk by the truncated series
    E un = dd[C - 1];
#pragma unroll
    for (int m = L - 1; m >= 0; --m) un = F::chain(Bb, un, dd[C - 1 - L + m]);
    const int ebase = j0 - L;
    const bool bulk = ebase >= head;
#pragma unroll
    for (int u = C - 1; u >= 0; --u) {
      if (u < C - 1) {
        const E dv = u >= L ? dd[u >= L ? u - L : 0] : tail[u < L ? u : 0];
        const int e = ebase + u;
        const E b = (!bulk && e >= 0 && e < head) ? __ldg(B + e) : Bb;
        un = F::chain(b, un, dv);
      }
      ob[lane * kXS + u] = un;
    }
#pragma unroll
    for (int q = 0; q < L; ++q) tail[q] = dd[C - L + q];
    __syncwarp();
    // coalesced store of the finished elements e = ebase + lane of every row
    {
      const int e = ebase + lane;
      if (e >= 0 && e < nx)
        for (int q = 0; q < rows; ++q) field[(size_t)q * P + e] = ob[q * kXS + lane];
    }
    __syncwarp();
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------- x sweep, banded operator

// The CN solve of a line is linear, u = T v with T = (I + aK)^{-1} (I - aK) and K the
// second difference with zero ghosts at -1 and n.  Reflection principle: extend v to
// the whole line as the odd function about both ghosts (v~_{-1-m} = -v~_{-1+m},
// v~_{n+m} = -v~_{n-m}); the free-line CN operator T_inf maps it to a function with
// the same symmetry, hence zero at the ghosts, which therefore solves the zero-ghost
// system: u_i = sum_k w_k v~_{i+k} with w the (symmetric) row of T_inf.  Its entries
// decay like rho^|k| (rho the root of rho + 1/rho = (1+2a)/a inside the unit circle),
// so in FP32 the sum stops at |k| <= W: the host takes w from an FP64 Thomas solve on
// a long line and picks the smallest W in {3, 5, 8} whose neglected entries sum to at
// most 2^-28.  Every output is then the same (2W+1)-tap dot product (weights in the
// kernel parameters), with no recurrence and no per-index coefficients: all the
// elements of a row are computed at once.  The centre weight is stored as w_0 - 1 and
// the identity part added last, u_j = v_j + [(w_0 - 1) v_j + sum_k w_k (v_{j-k} +
// v_{j+k})]: the bracket is small (|w_0 - 1| and |w_k| are O(a)), so rounding the
// weights to FP32 perturbs u far below an FP32 ulp of it, and the same perturbation,
// repeated every step, does not build up a drift.
//
// Each warp owns band_rows consecutive rows (the host sizes this so that all warps
// are resident at once) and works on them alone, with warp barriers only.  A row
// arrives by one bulk copy into a shared-memory slot with kBandPad elements of room
// on both sides; band_stages rows are in flight per warp.  Lane l serves the 16-byte
// vectors l, l + 32, ... of the row (EPT elements each).  Per row: the pending scale
// and the pointwise substep in place; then the odd images of the first and last 7
// elements into the pads and zero at the ghosts; then the dot products from 16-byte
// shared loads, stored straight to the field (in place: a warp owns its rows).
// Needs nx >= kBandPad so that one reflection covers every window.
constexpr int kBandPad = 8;     // room for the odd images on each side of a row slot

__device__ __forceinline__ float shfl_e(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float2 shfl_e(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float shfl_up_e(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float2 shfl_up_e(float2 v, int d) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float shfl_down_e(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float2 shfl_down_e(float2 v, int d) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// What one warp of the banded x sweep works on: nrow consecutive rows from row0 of
// one field, taken G rows at a time (a group), streamed through S shared-memory
// stages of G row slots of slot_elems elements each.
template <class E> struct XRows {
  E* field;
  const float4* fx;      // trap factors along x, [pitch] (16-byte vectors)
  const E* fyz;          // trap factor per row
  const E* wt;           // w_{k-W}, k = 0 .. 2W (centre as w_0 - 1)
  const double* scale;   // pending renormalisation factor
  const unsigned int* step_ctr;   // the step counter behind its dither (null: none)
  int* status;
  unsigned long long wait_ns;   // limit of the first bounded wait on each row copy
  long long row0;
  int nrow, nx, pitch, S, G, slot_elems;
  int pw;                // 1: pointwise substep on load; 0: only the pending factor
  float dtg;             // dt g
};

// Barriers and ghost -1 of a warp's row slots (before the dependent-launch wait).
template <class E>
__device__ __forceinline__ void x_band_init(uint64_t* full, E* slots, int S, int nslots,
                                            int slot_elems) {
  const int lane = threadIdx.x & 31;
  if (lane == 0)
    for (int q = 0; q < S; ++q) mbar_init(&full[q], 1);
  for (int q = lane; q < nslots; q += 32) slots[(size_t)q * slot_elems - 1] = E{};   // ghost -1
  __syncwarp();
}

template <class R, bool CPLX, int W>
__device__ __forceinline__ void x_band_rows(const XRows<typename Field<R, CPLX>::E>& a,
                                            uint64_t* full, typename Field<R, CPLX>::E* slots) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  constexpr int EPT = 16 / (int)sizeof(E);   // elements per 16-byte vector
  constexpr int H = (W + EPT - 1) / EPT;     // halo vectors on each side of a window
  constexpr int NV = 2 * H + 1;              // vectors in a window
  static_assert(H * EPT <= kBandPad, "window inside the slot");
  const int nx = a.nx, pitch = a.pitch, S = a.S, G = a.G, nrow = a.nrow, se = a.slot_elems;
  const int lane = threadIdx.x & 31;
  const int nvec = (nx + EPT - 1) / EPT;
  const float inv_nvec = 1.0f / (float)nvec;
  const int ngroups = (nrow + G - 1) / G;
  const long long row0 = a.row0;
  E* field = a.field;
  E wt[W + 1];   // wt[0] = w_0 - 1, wt[k] = w_k
#pragma unroll
  for (int k = 0; k <= W; ++k) wt[k] = a.wt[W + k];
  const float4* fx = a.fx;
  const E* fyz = a.fyz;
  const uint32_t rowbytes = (uint32_t)((size_t)pitch * sizeof(E));
  const R dtg = (R)a.dtg;
  // row slot r of stage st
  auto slot_of = [&](int st, int r) { return slots + (size_t)(st * G + r) * se; };
  auto issue = [&](int i, int st) {   // group i of this warp -> stage st = i mod S, one bulk copy per row
    const int rows = min(G, nrow - i * G);
    mbar_arrive_expect_tx(&full[st], (uint32_t)rows * rowbytes);
    for (int r = 0; r < rows; ++r)
      bulk_load(slot_of(st, r), field + (size_t)(row0 + (long long)i * G + r) * pitch, rowbytes,
                &full[st]);
  };
  if (lane == 0)
    for (int i = 0; i < S && i < ngroups; ++i) issue(i, i);
  // the pending factor, formed after the first copies are out (its loads' latency
  // overlaps theirs)
  const R s = (R)(*a.scale) * (R)step_dither_f(a.step_ctr);
  // trap factor of row `lane` of the current group, loaded one group ahead; a lane
  // takes its row's factor from lane r by shuffle
  E fcur = lane < min(G, nrow) ? fyz[row0 + lane] : F::zero();

  int st = 0;
  uint32_t phase = 0;
  for (int i = 0; i < ngroups; ++i) {
    const int rows = min(G, nrow - i * G);
    const int nv = rows * nvec;            // vectors of the group
    const long long gr0 = row0 + (long long)i * G;
    const E fnext = (i + 1 < ngroups && lane < min(G, nrow - (i + 1) * G)) ? fyz[gr0 + G + lane] : F::zero();
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[st], phase, a.wait_ns))) {
      if (lane == 0) {
        atomicOr(a.status, kStatusTimeout);
        // wait (bounded) for every copy still in flight before the warp exits
        for (int q = i; q < i + S && q < ngroups; ++q)
          mbar_wait_bounded(&full[q % S], (uint32_t)(q / S) & 1u, kWaitLimitNs);
      }
      __syncwarp();
      return;
    }
    // pointwise substep in place (past nx too: overwritten below); lanes run over the
    // group's (row, vector) pairs and take the polynomial branch together when every
    // argument of the warp allows it
    for (int v0 = 0; v0 < nv; v0 += 32) {
      const int idx = v0 + lane;
      const bool act = idx < nv;
      const int r = act ? (G == 1 ? 0 : __float2int_rz(((float)idx + 0.5f) * inv_nvec)) : 0;
      const int v = act ? idx - r * nvec : 0;
      float4* vp = reinterpret_cast<float4*>(slot_of(st, r) + v * EPT);
      float4 raw = *vp;
      const float4 fxv = __ldg(fx + v);
      const E fr = shfl_e(fcur, r);
      E* ev = reinterpret_cast<E*>(&raw);
      const E* fe = reinterpret_cast<const E*>(&fxv);
      R y[EPT];
      R ymax = R(0);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        ev[e] = F::scaled(ev[e], s);
        y[e] = dtg * F::abs2(ev[e]);
        ymax = fmaxf(ymax, fabsf(y[e]));
      }
      if (!a.pw) {
        // kinetic-only step: the pending factor alone
      } else if (__all_sync(0xffffffffu, !act || ymax <= R(0.0625))) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) ev[e] = F::nonlinear_small(ev[e], F::mul(fe[e], fr), y[e]);
      } else {
#pragma unroll
        for (int e = 0; e < EPT; ++e) ev[e] = F::nonlinear_full(ev[e], F::mul(fe[e], fr), y[e]);
      }
      if (act) *vp = raw;
    }
    __syncwarp();
    // per row: odd images about -1 (positions -2..-8) and about nx (nx+1..nx+7), and
    // the ghost nx: 15 tasks
    for (int t = lane; t < 15 * rows; t += 32) {
      const int r = t / 15, k = t - 15 * r;
      E* row = slot_of(st, r);
      // k < 7: -row[k] -> -2-k; k < 14: -row[nx-1-m] -> nx+1+m; k = 14: -row[-1] (= 0)
      // -> nx, the ghost (a signed zero, which leaves every sum unchanged)
      const int src = k < 7 ? k : k < 14 ? nx - 1 - (k - 7) : -1;
      const int dst = k < 7 ? -2 - k : k < 14 ? nx + 1 + (k - 7) : nx;
      row[dst] = F::scaled(row[src], R(-1));
    }
    __syncwarp();
    for (int idx = lane; idx < nv; idx += 32) {
      const int r = G == 1 ? 0 : __float2int_rz(((float)idx + 0.5f) * inv_nvec);
      const int v = idx - r * nvec;
      const int x0 = v * EPT;
      const float4* src = reinterpret_cast<const float4*>(slot_of(st, r) + x0 - H * EPT);
      float4 wv[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) wv[q] = src[q];
      const E* win = reinterpret_cast<const E*>(wv);
      float4 ov;
      E* o = reinterpret_cast<E*>(&ov);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int c = H * EPT + e;   // the output's position in the window
        E acc = F::mul(wt[0], win[c]);
#pragma unroll
        for (int k = 1; k <= W; ++k) acc = F::chain(wt[k], F::add(win[c - k], win[c + k]), acc);
        o[e] = F::add(win[c], acc);
      }
      E* grow = field + (size_t)(gr0 + r) * pitch;
      if (x0 + EPT <= nx) {
        *reinterpret_cast<float4*>(grow + x0) = ov;
      } else {
#pragma unroll
        for (int e = 0; e < EPT; ++e)
          if (x0 + e < nx) grow[x0 + e] = o[e];
      }
    }
    __syncwarp();
    if (lane == 0 && i + S < ngroups) {
      fence_smem_to_async();
      issue(i + S, st);
    }
    fcur = fnext;
    if (++st == S) {
      st = 0;
      phase ^= 1u;
    }
  }
}

// One row at a time (rows of 32 or more 16-byte vectors fill the lanes by themselves).
// Per-row work is kept to the copy, the wait and the images: the stage and its phase
// advance by counting, the trap factors along x of the lane's first NC vectors stay
// in registers (they are the same in every row), the band weights too, and the first
// NC passes over a row are unrolled.
template <class R, bool CPLX, int W>
__device__ __forceinline__ void x_band_rows_single(const XRows<typename Field<R, CPLX>::E>& a,
                                            uint64_t* full, typename Field<R, CPLX>::E* slots) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  constexpr int EPT = 16 / (int)sizeof(E);   // elements per 16-byte vector
  constexpr int H = (W + EPT - 1) / EPT;     // halo vectors on each side of a window
  constexpr int NV = 2 * H + 1;              // vectors in a window
  constexpr int NC = 2;                      // 32-lane passes with cached trap factors
  static_assert(H * EPT <= kBandPad, "window inside the slot");
  const int nx = a.nx, pitch = a.pitch, S = a.S, nrow = a.nrow, se = a.slot_elems;
  const int lane = threadIdx.x & 31;
  const int nvec = (nx + EPT - 1) / EPT;
  E* field = a.field;
  const float4* fx = a.fx;
  const uint32_t rowbytes = (uint32_t)((size_t)pitch * sizeof(E));
  E* gsrc = field + (size_t)a.row0 * pitch;   // row i + S's copy source
  if (lane == 0)
    for (int i = 0; i < S && i < nrow; ++i) {
      mbar_arrive_expect_tx(&full[i], rowbytes);
      bulk_load(slots + (size_t)i * se, gsrc, rowbytes, &full[i]);
      gsrc += pitch;
    }
  E wt[W + 1];   // wt[0] = w_0 - 1, wt[k] = w_k
#pragma unroll
  for (int k = 0; k <= W; ++k) wt[k] = a.wt[W + k];
  float4 fxc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c)
    fxc[c] = lane + 32 * c < nvec ? __ldg(fx + lane + 32 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
  // (formed after the first copies are out: its loads' latency overlaps theirs)
  const R s = (R)(*a.scale) * (R)step_dither_f(a.step_ctr);
  const R dtg = (R)a.dtg;
  const bool pw = a.pw != 0;
  const E* fyz = a.fyz + a.row0;
  E f_next = fyz[0];
  E* grow = field + (size_t)a.row0 * pitch;   // row i's output
  int st = 0;
  uint32_t phase = 0;

  // pointwise substep of vector v (lanes past the row idle but vote)
  auto point = [&](E* row, int v, float4 fxv, E fr) {
    const bool act = v < nvec;
    float4* vp = reinterpret_cast<float4*>(row + (act ? v : 0) * EPT);
    float4 raw = *vp;
    E* ev = reinterpret_cast<E*>(&raw);
    const E* fe = reinterpret_cast<const E*>(&fxv);
    R y[EPT];
    R ymax = R(0);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      ev[e] = F::scaled(ev[e], s);
      y[e] = dtg * F::abs2(ev[e]);
      ymax = fmaxf(ymax, fabsf(y[e]));
    }
    if (!pw) {
      // kinetic-only step: the pending factor alone
    } else if (__all_sync(0xffffffffu, !act || ymax <= R(0.0625))) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) ev[e] = F::nonlinear_small(ev[e], F::mul(fe[e], fr), y[e]);
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) ev[e] = F::nonlinear_full(ev[e], F::mul(fe[e], fr), y[e]);
    }
    if (act) *vp = raw;
  };
  // banded operator at vector v of the row, stored to the field
  auto band = [&](const E* row, int v) {
    const int x0 = v * EPT;
    const float4* src = reinterpret_cast<const float4*>(row + x0 - H * EPT);
    float4 wv[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) wv[q] = src[q];
    const E* win = reinterpret_cast<const E*>(wv);
    float4 ov;
    E* o = reinterpret_cast<E*>(&ov);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int c = H * EPT + e;   // the output's position in the window
      E acc = F::mul(wt[0], win[c]);
#pragma unroll
      for (int k = 1; k <= W; ++k) acc = F::chain(wt[k], F::add(win[c - k], win[c + k]), acc);
      o[e] = F::add(win[c], acc);
    }
    if (x0 + EPT <= nx) {
      *reinterpret_cast<float4*>(grow + x0) = ov;
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (x0 + e < nx) grow[x0 + e] = o[e];
    }
  };

  for (int i = 0; i < nrow; ++i) {
    E* row = slots + (size_t)st * se;
    const E fr = f_next;
    if (i + 1 < nrow) f_next = fyz[i + 1];
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[st], phase, a.wait_ns))) {
      if (lane == 0) {
        atomicOr(a.status, kStatusTimeout);
        // wait (bounded) for every copy still in flight before the warp exits
        for (int q = i; q < i + S && q < nrow; ++q)
          mbar_wait_bounded(&full[q % S], (uint32_t)(q / S) & 1u, kWaitLimitNs);
      }
      __syncwarp();
      return;
    }
    // pointwise substep in place (past nx too: overwritten below); the lanes of a
    // warp take the polynomial branch together when every argument allows it
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (32 * c < nvec) point(row, lane + 32 * c, fxc[c], fr);
    for (int v0 = 32 * NC; v0 < nvec; v0 += 32)
      point(row, v0 + lane, __ldg(fx + min(v0 + lane, nvec - 1)), fr);
    __syncwarp();
    // odd images about -1 (positions -2..-8) and about nx (nx+1..nx+7), and the ghost
    // nx as -row[-1] (a signed zero, which leaves every sum unchanged): one predicated
    // load / negate / store per lane
    if (lane < 15) {
      const int src = lane < 7 ? lane : lane < 14 ? nx - 1 - (lane - 7) : -1;
      const int dst = lane < 7 ? -2 - lane : lane < 14 ? nx + 1 + (lane - 7) : nx;
      row[dst] = F::scaled(row[src], R(-1));
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (lane + 32 * c < nvec) band(row, lane + 32 * c);
    for (int v = lane + 32 * NC; v < nvec; v += 32) band(row, v);
    __syncwarp();
    if (lane == 0 && i + S < nrow) {
      fence_smem_to_async();
      mbar_arrive_expect_tx(&full[st], rowbytes);
      bulk_load(row, gsrc, rowbytes, &full[st]);
      gsrc += pitch;
    }
    grow += pitch;
    if (++st == S) {
      st = 0;
      phase ^= 1u;
    }
  }
}

template <class R, bool CPLX, int W, bool GROUPED>
__global__ void __launch_bounds__(32 * kBandWarps) k_sweep_x_band(const __grid_constant__ SweepParams p) {
  using E = typename Field<R, CPLX>::E;
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = p.band_stages, G = p.band_group, slot_elems = p.pitch + 2 * kBandPad;
  const int wib = threadIdx.x >> 5;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem) + wib * S;
  E* slots = reinterpret_cast<E*>(smem + 128 * kBandWarps) + (size_t)wib * S * G * slot_elems + kBandPad;
  const long long nrows = (long long)p.ny * p.nz;
  // rows in equal shares (band_rows or band_rows + 1 per warp): every SM the same work
  const int w = blockIdx.x * kBandWarps + wib;
  const long long row0 = (long long)w * p.band_rows + min(w, p.band_rem);
  const int nrow = (int)max(0LL, min((long long)p.band_rows + (w < p.band_rem ? 1 : 0), nrows - row0));
  x_band_init(full, slots, S, S * G, slot_elems);
  pdl_begin();
  // the pending factor (see k_sweep_x_reg), for every warp of the block
  __shared__ double s_factor;
  const bool defer = p.norm_defer != 0;
  if (defer) {
    const double f = deferred_scale(p.partials + (size_t)(blockIdx.x % p.norm_copies) * p.norm_blocks,
                                    p.norm_blocks, p.dV, p.status, blockIdx.x == 0, p.scale_state, p.scale);
    if (threadIdx.x == 0) s_factor = f;
    __syncthreads();
  }
  if (nrow == 0) return;
  XRows<E> a;
  a.field = static_cast<E*>(p.psi);
  a.fx = static_cast<const float4*>(p.band_fx);
  a.fyz = static_cast<const E*>(p.band_fyz);
  a.wt = reinterpret_cast<const E*>(p.band_wt);
  a.scale = defer ? &s_factor : p.scale;
  a.step_ctr = p.step_ctr;
  a.status = p.status;
  a.wait_ns = p.wait_ns;
  a.row0 = row0;
  a.nrow = nrow;
  a.nx = p.nx;
  a.pitch = p.pitch;
  a.S = S;
  a.G = G;
  a.slot_elems = slot_elems;
  a.pw = p.pw;
  a.dtg = p.band_dtg;
  if (!GP_IN(row0 + nrow - 1, nrows, p.status)) return;
  if (GROUPED) x_band_rows<R, CPLX, W>(a, full, slots);
  else x_band_rows_single<R, CPLX, W>(a, full, slots);
}

// Banded x sweep with the row in registers, for rows of nx = 8 m <= 256 points and
// W <= 7: lane l owns the eight elements [8l, 8l + 8) of the warp's current row (two
// 16-byte vectors of a real field, four of a complex one), loaded coalesced with the
// next row's already in flight.  The pending factor and the pointwise substep are
// applied in registers; the W neighbours on each side come from lanes l - 1 and l + 1
// by shuffles, and at the row's ends the odd images (-v mirrored about the ghosts -1
// and nx, zero at the ghosts) come from the lane's own elements (8 >= W + 1).  No
// shared memory, copies or waits: the instructions per point are the arithmetic plus
// a few shuffles, which is what bounds the copy-fed kernel above.  Each warp works on
// a_rows consecutive rows; every warp of the launch is resident at once.
template <bool CPLX, int W>
__global__ void __launch_bounds__(32 * kXRegWarps) k_sweep_x_reg(const __grid_constant__ SweepParams p) {
  using F = Field<float, CPLX>;
  using E = typename F::E;
  constexpr int EPT = 16 / (int)sizeof(E);   // elements per 16-byte vector
  constexpr int VPL = 8 / EPT;               // vectors per lane
  static_assert(W <= 7, "images from the lane's own eight elements");
  const int lane = threadIdx.x & 31;
  const long long nrows = (long long)p.ny * p.nz;
  // rows in equal shares (band_rows or band_rows + 1 per warp): every SM the same work
  const int w = blockIdx.x * kXRegWarps + (threadIdx.x >> 5);
  const long long row0 = (long long)w * p.band_rows + min(w, p.band_rem);
  const int nrow = (int)max(0LL, min((long long)p.band_rows + (w < p.band_rem ? 1 : 0), nrows - row0));
  const int nx = p.nx, pitch = p.pitch;
  const int x0 = 8 * lane;
  const bool act = x0 < nx;                  // lanes past the row hold zeros
  const bool first = lane == 0, last = x0 + 8 == nx;
  E wt[W + 1];   // wt[0] = w_0 - 1, wt[k] = w_k
#pragma unroll
  for (int k = 0; k <= W; ++k) wt[k] = reinterpret_cast<const E*>(p.band_wt)[W + k];
  E fx[8];
  {
    const float4* fxv = reinterpret_cast<const float4*>(static_cast<const E*>(p.band_fx) + x0);
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
      const float4 f = act ? __ldg(fxv + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int e = 0; e < EPT; ++e) fx[q * EPT + e] = reinterpret_cast<const E*>(&f)[e];
    }
  }
  pdl_begin();
  const float dtg = p.band_dtg;
  const bool pw = p.pw != 0;
  E* field = static_cast<E*>(p.psi);
  const E* fyz = static_cast<const E*>(p.band_fyz);
  const long long nel = nrows * pitch;   // field elements (bounds checks)
  auto load_row = [&](long long r, float4 (&buf)[VPL]) {
    const float4* src = reinterpret_cast<const float4*>(field + (size_t)r * pitch + x0);
#pragma unroll
    for (int q = 0; q < VPL; ++q)
      buf[q] = act && GP_IN(r * pitch + x0 + (q + 1) * EPT - 1, nel, p.status)
                   ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  float s = 1.f;   // the pending factor, set below once the first row's loads are out
  // row r's pointwise substep, banded operator and store, from its loaded vectors
  auto process = [&](long long r, const float4 (&cur)[VPL], E fr) {
    E v[8];
#pragma unroll
    for (int q = 0; q < VPL; ++q)
#pragma unroll
      for (int e = 0; e < EPT; ++e) v[q * EPT + e] = reinterpret_cast<const E*>(&cur[q])[e];
    // pending factor and pointwise substep (the warp takes the polynomial branch when
    // every argument allows it)
    float y[8];
    float ymax = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = F::scaled(v[e], s);
      y[e] = dtg * F::abs2(v[e]);
      ymax = fmaxf(ymax, fabsf(y[e]));
    }
    if (!pw) {
    } else if (__all_sync(0xffffffffu, ymax <= 0.0625f)) {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = F::nonlinear_small(v[e], F::mul(fx[e], fr), y[e]);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = F::nonlinear_full(v[e], F::mul(fx[e], fr), y[e]);
    }
    // halo: lo[m] = position x0 - m, hi[m] = position x0 + 7 + m (m = 1..W)
    E lo[W + 1], hi[W + 1];
#pragma unroll
    for (int m = 1; m <= W; ++m) {
      lo[m] = shfl_up_e(v[8 - m], 1);
      hi[m] = shfl_down_e(v[m - 1], 1);
      // odd images: position -m is 0 (m = 1) or -v[m - 2]; position nx - 1 + m is 0
      // (m = 1) or -v[9 - m]
      if (first) lo[m] = m == 1 ? F::zero() : F::scaled(v[m - 2], -1.f);
      if (last) hi[m] = m == 1 ? F::zero() : F::scaled(v[9 - m], -1.f);
    }
    auto win = [&](int j) -> E { return j < 0 ? lo[-j] : (j >= 8 ? hi[j - 7] : v[j]); };
    E o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      E acc = F::mul(wt[0], v[e]);
#pragma unroll
      for (int k = 1; k <= W; ++k) acc = F::chain(wt[k], F::add(win(e - k), win(e + k)), acc);
      o[e] = F::add(v[e], acc);
    }
    if (act && GP_IN(r * pitch + x0 + 7, nel, p.status)) {
      float4* dst = reinterpret_cast<float4*>(field + (size_t)r * pitch + x0);
#pragma unroll
      for (int q = 0; q < VPL; ++q) dst[q] = *reinterpret_cast<const float4*>(&o[q * EPT]);
    }
  };
  // the next row's loads are in flight while a row is processed (deeper prefetch,
  // in registers or through shared memory, measured slower at 240 x 200 x 160);
  // the first row's loads go out before the pending factor is known: it is stored, or
  // summed from the previous z sweep's partials (every block the same bits; all
  // threads take part before any warp may leave)
  float4 cur[VPL], nxt[VPL];
  E fr = F::zero();
  if (nrow > 0) {
    load_row(row0, cur);
    fr = fyz[row0];
  }
  {
    // one thread forms the factor with the step's dither (FP64 arithmetic is slow on
    // this part), the block shares it
    __shared__ float s_block;
    const double f = p.norm_defer
                         ? deferred_scale(p.partials + (size_t)(blockIdx.x % p.norm_copies) * p.norm_blocks,
                                          p.norm_blocks, p.dV, p.status, blockIdx.x == 0, p.scale_state, p.scale)
                         : 0.0;
    if (threadIdx.x == 0) s_block = (float)((p.norm_defer ? f : *p.scale) * step_dither(p.step_ctr));
    __syncthreads();
    s = s_block;
  }
  if (nrow == 0) return;
  for (int i = 0; i < nrow; ++i) {
    const long long r = row0 + i;
    E frn = fr;
    if (i + 1 < nrow) {
      load_row(r + 1, nxt);
      frn = fyz[r + 1];
    }
    process(r, cur, fr);
#pragma unroll
    for (int q = 0; q < VPL; ++q) cur[q] = nxt[q];
    fr = frn;
  }
}

// Batched x sweep: warp w of the launch takes work item w (rows of one slot).
template <class R, bool CPLX, int W>
__global__ void __launch_bounds__(32 * kBatchXWarps) k_batch_x_band(const __grid_constant__ BatchArgs b) {
  using E = typename Field<R, CPLX>::E;
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = b.stages, GM = b.group_max, slot_elems = b.slot_elems;
  const int wib = threadIdx.x >> 5;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem) + wib * S;
  const int w = blockIdx.x * kBatchXWarps + wib;
  // the item's G rows of a stage sit in its first G of the GM slots per stage
  const int G = w < b.nitems ? static_cast<const XItem*>(b.items)[w].group : 1;
  E* slots = reinterpret_cast<E*>(smem + 128 * kBatchXWarps) + (size_t)wib * S * GM * slot_elems + kBandPad;
  x_band_init(full, slots, S, S * G, slot_elems);
  pdl_begin();
  if (w >= b.nitems) return;
  const XItem it = static_cast<const XItem*>(b.items)[w];
  const SlotDesc& d = b.slots[it.slot];
  XRows<E> a;
  a.field = static_cast<E*>(d.field);
  a.fx = static_cast<const float4*>(d.fx);
  a.fyz = static_cast<const E*>(d.fyz);
  a.wt = reinterpret_cast<const E*>(d.wt[0]) + (kBandHalfMax - W);
  a.scale = d.scale;
  a.step_ctr = nullptr;
  a.status = b.status;
  a.wait_ns = b.wait_ns;
  a.row0 = it.row0;
  a.nrow = it.nrow;
  a.nx = d.nx;
  a.pitch = d.pitch;
  a.S = S;
  a.G = G;
  a.slot_elems = slot_elems;
  a.pw = 1;
  a.dtg = d.dtg;
  x_band_rows<R, CPLX, W>(a, full, slots);
}

// Batched x sweep with rows in registers, for slots whose rows are nx = EPL m points,
// at most 32 EPL (half-width W <= 7): EPL = 16 real or 8 complex elements per lane, four
// 16-byte vectors.  Lane li of a row owns its elements [EPL li, EPL li + EPL).  Warp w
// takes work item w, it.nrow consecutive rows of one slot, it.group = floor(32 / L)
// rows at a time (L = nx / EPL lanes per row); the next pass's rows are in flight while
// a pass is processed.  Per row as in k_sweep_x_reg: pending factor and pointwise
// substep in registers, the W neighbours by shuffles from lanes li -/+ 1, odd images at
// the row's own first and last lanes.  The pointwise polynomial is chosen per row (a
// ballot over the row's lanes), so a slot's arithmetic does not depend on which rows
// share a warp, and the operations are those of the copy-fed kernel (x_band_rows) in
// the same order.
template <bool CPLX, int W>
__global__ void __launch_bounds__(32 * kXRegWarps) k_batch_x_reg(const __grid_constant__ BatchArgs b) {
  using F = Field<float, CPLX>;
  using E = typename F::E;
  constexpr int EPT = 16 / (int)sizeof(E);   // elements per 16-byte vector
  constexpr int VPL = 4, EPL = VPL * EPT;    // vectors and elements per lane
  static_assert(W <= 7, "images from the lane's own elements");
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * kXRegWarps + (threadIdx.x >> 5);
  pdl_begin();
  if (w >= b.nitems) return;
  const XItem it = static_cast<const XItem*>(b.items)[w];
  const SlotDesc& d = b.slots[it.slot];
  const int nx = d.nx, pitch = d.pitch;
  const int L = nx / EPL, RP = it.group;     // lanes per row, rows per pass
  const int rp = lane / L, li = lane - rp * L;
  const bool lane_on = rp < RP;
  const bool first = li == 0, last = li == L - 1;
  const int x0 = EPL * li;
  const unsigned int row_mask = !lane_on ? 0u : (L >= 32 ? 0xffffffffu : ((1u << L) - 1u) << (rp * L));
  E wt[W + 1];   // wt[0] = w_0 - 1, wt[k] = w_k
  {
    const E* wsrc = reinterpret_cast<const E*>(d.wt[0]) + (kBandHalfMax - W);
#pragma unroll
    for (int k = 0; k <= W; ++k) wt[k] = wsrc[W + k];
  }
  E fx[EPL];
  {
    const float4* fxv = reinterpret_cast<const float4*>(static_cast<const E*>(d.fx) + x0);
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
      const float4 f = lane_on ? __ldg(fxv + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int e = 0; e < EPT; ++e) fx[q * EPT + e] = reinterpret_cast<const E*>(&f)[e];
    }
  }
  const float s = (float)(*d.scale);
  const float dtg = d.dtg;
  E* field = static_cast<E*>(d.field);
  const E* fyz = static_cast<const E*>(d.fyz);
  const long long nel = (long long)d.ny * d.nz * pitch;
  const int npass = (it.nrow + RP - 1) / RP;
  auto row_of = [&](int q) { return it.row0 + (long long)q * RP + rp; };
  auto valid = [&](int q) { return lane_on && q * RP + rp < it.nrow; };
  auto load_row = [&](int q, float4 (&buf)[VPL]) {
    const long long r = row_of(q);
    const bool ok = valid(q) && GP_IN(r * pitch + x0 + EPL - 1, nel, b.status);
    const float4* src = reinterpret_cast<const float4*>(field + (size_t)(ok ? r : 0) * pitch + x0);
#pragma unroll
    for (int qq = 0; qq < VPL; ++qq) buf[qq] = ok ? src[qq] : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  float4 cur[VPL], nxt[VPL];
  load_row(0, cur);
  E fr = valid(0) ? fyz[row_of(0)] : F::zero();
  for (int q = 0; q < npass; ++q) {
    E frn = fr;
    if (q + 1 < npass) {
      load_row(q + 1, nxt);
      frn = valid(q + 1) ? fyz[row_of(q + 1)] : F::zero();
    }
    E v[EPL];
#pragma unroll
    for (int qq = 0; qq < VPL; ++qq)
#pragma unroll
      for (int e = 0; e < EPT; ++e) v[qq * EPT + e] = F::scaled(reinterpret_cast<const E*>(&cur[qq])[e], s);
    // (the argument dt g |v|^2 is formed again where it is used rather than held)
    float ymax = 0.f;
#pragma unroll
    for (int e = 0; e < EPL; ++e) ymax = fmaxf(ymax, fabsf(dtg * F::abs2(v[e])));
    // the row takes the polynomial when every argument of its lanes allows it
    const unsigned int big = __ballot_sync(0xffffffffu, ymax > 0.0625f || !(ymax == ymax));
    if ((big & row_mask) == 0u) {
#pragma unroll
      for (int e = 0; e < EPL; ++e) v[e] = F::nonlinear_small(v[e], F::mul(fx[e], fr), dtg * F::abs2(v[e]));
    } else {
#pragma unroll
      for (int e = 0; e < EPL; ++e) v[e] = F::nonlinear_full(v[e], F::mul(fx[e], fr), dtg * F::abs2(v[e]));
    }
    // halo: lo[m] = position x0 - m, hi[m] = position x0 + EPL - 1 + m (m = 1..W); odd
    // images: position -m is 0 (m = 1) or -v[m - 2], position nx - 1 + m is 0 (m = 1)
    // or -v[EPL + 1 - m]
    E lo[W + 1], hi[W + 1];
#pragma unroll
    for (int m = 1; m <= W; ++m) {
      lo[m] = shfl_up_e(v[EPL - m], 1);
      hi[m] = shfl_down_e(v[m - 1], 1);
      if (first) lo[m] = m == 1 ? F::zero() : F::scaled(v[m - 2], -1.f);
      if (last) hi[m] = m == 1 ? F::zero() : F::scaled(v[EPL + 1 - m], -1.f);
    }
    auto win = [&](int j) -> E { return j < 0 ? lo[-j] : (j >= EPL ? hi[j - EPL + 1] : v[j]); };
    const long long r = row_of(q);
    const bool store = valid(q) && GP_IN(r * pitch + x0 + EPL - 1, nel, b.status);
    float4* dst = reinterpret_cast<float4*>(field + (size_t)(store ? r : 0) * pitch + x0);
#pragma unroll
    for (int qq = 0; qq < VPL; ++qq) {
      float4 ov;
      E* o = reinterpret_cast<E*>(&ov);
#pragma unroll
      for (int t = 0; t < EPT; ++t) {
        const int e = EPT * qq + t;
        E acc = F::mul(wt[0], v[e]);
#pragma unroll
        for (int k = 1; k <= W; ++k) acc = F::chain(wt[k], F::add(win(e - k), win(e + k)), acc);
        o[t] = F::add(v[e], acc);
      }
      if (store) dst[qq] = ov;
    }
#pragma unroll
    for (int qq = 0; qq < VPL; ++qq) cur[qq] = nxt[qq];
    fr = frn;
  }
}

// y (AXIS 1) or z (AXIS 2) sweep as the banded operator on the odd extension (see the
// x sweep above), for the FP32 field.  Thread t owns the 16-byte vector
// xv = t mod nvec (EPT consecutive x) of one segment of band_seg points of one line;
// consecutive threads are consecutive x, so every load and store is coalesced.  The
// segment's outputs need its inputs plus W on each side (odd images past the line's
// ends), held in a ring of P = 2W+1 vectors: the loop is unrolled by P, so the ring
// slot of every tap is a compile-time constant; the P new inputs of a turn are loaded
// together at its start, so that they are in flight at once.  Out of place (p.psi -> p.out):
// neighbouring segments read each other's inputs.  With NORM the block also sums
// |u|^2 (FP32 within a ring turn, FP64 across) and the last block turns the partials
// into the renormalisation factor.
// What one thread of a banded y / z sweep works on.
template <class E> struct LineArgs {
  const E* psi;          // input field, [nz][ny][pitch]
  E* out;                // output field, same layout
  const E* wt;           // w_{k-W}, k = 0 .. 2W (centre as w_0 - 1)
  int nx, ny, nz, n, pitch, Ls;
  int* status;           // bounds checks of GP_CHECK builds
};

// Thread t's segment of one line; returns the sum of |u|^2 it stored (NORM): FP32 within
// a turn, float-float across turns.
template <class R, bool CPLX, int AXIS, bool NORM, int W>
__device__ __forceinline__ FF band_line_thread(const LineArgs<typename Field<R, CPLX>::E>& p,
                                                   long long t) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  constexpr int EPT = 16 / (int)sizeof(E);
  constexpr int P = 2 * W + 1;
  const int nx = p.nx, n = p.n, Ls = p.Ls;
  const int nvec = (nx + EPT - 1) / EPT;
  const int nother = AXIS == 1 ? p.nz : p.ny;
  const int nseg = (n + Ls - 1) / Ls;
  const E* wt = p.wt;
  FF acc = FF{0.f, 0.f};
  if (t < (long long)nvec * nother * nseg) {
    // t < nvec * nother * nseg <= 1024 * 2048 * 293 < 2^31 (extents <= 2048, segments
    // of at least 2W + 1 >= 7 points): 32-bit division, not 64-bit
    const unsigned int tu = (unsigned int)t;
    const int xv = (int)(tu % (unsigned int)nvec);
    const unsigned int rest = tu / (unsigned int)nvec;
    const int o = (int)(rest % (unsigned int)nother), sg = (int)(rest / (unsigned int)nother);
    const size_t pitch = (size_t)p.pitch;
    const size_t base = (AXIS == 1 ? (size_t)o * p.ny * pitch : (size_t)o * pitch) + (size_t)xv * EPT;
    const float4* in = reinterpret_cast<const float4*>(p.psi + base);
    float4* out = reinterpret_cast<float4*>(p.out + base);
    const size_t sv = (AXIS == 1 ? pitch : pitch * p.ny) * sizeof(E) / 16;   // line stride in vectors
    const int valid = min(EPT, nx - xv * EPT);   // elements of this vector inside the field
    const int j0 = sg * Ls, j1 = min(n, j0 + Ls);
    const bool interior = j0 >= W && j0 + Ls + W <= n;
    // input j of the odd extension about the ghosts -1 and n
    // 16-byte vectors of the field, and this line's first one (bounds checks)
    const long long nvec_all = (long long)p.nz * p.ny * (long long)pitch / EPT, v0 = (long long)(base / EPT);
    auto ld = [&](int j) -> float4 {
      if (interior || (j >= 0 && j < n))
        return GP_IN(v0 + (long long)j * sv, nvec_all, p.status) ? in[(size_t)j * sv]
                                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      if (j == -1 || j == n) return make_float4(0.f, 0.f, 0.f, 0.f);
      const int m = j < 0 ? -2 - j : 2 * n - j;
      const float4 v = GP_IN(v0 + (long long)m * sv, nvec_all, p.status) ? in[(size_t)m * sv]
                                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
      return make_float4(-v.x, -v.y, -v.z, -v.w);
    };
    float4 ring[P];
#pragma unroll
    for (int m = 0; m < 2 * W; ++m) ring[m] = ld(j0 - W + m);
    for (int b = j0; b < j1; b += P) {
      float part = 0.f;
      // the turn's P new inputs, all in flight before the first output needs one
      float4 nv[P];
#pragma unroll
      for (int u = 0; u < P; ++u)
        nv[u] = (interior || b + u < j1) ? ld(b + u + W) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int j = b + u;
        if (interior || j < j1) {
          ring[(u + 2 * W) % P] = nv[u];
          const E* c = reinterpret_cast<const E*>(&ring[(u + W) % P]);
          float4 ov;
          E* oe = reinterpret_cast<E*>(&ov);
#pragma unroll
          for (int e = 0; e < EPT; ++e) {
            E a = F::mul(wt[W], c[e]);
#pragma unroll
            for (int k = 1; k <= W; ++k) {
              const E* lo = reinterpret_cast<const E*>(&ring[(u + W - k) % P]);
              const E* hi = reinterpret_cast<const E*>(&ring[(u + W + k) % P]);
              a = F::chain(wt[W + k], F::add(lo[e], hi[e]), a);
            }
            oe[e] = F::add(c[e], a);
          }
          if (!GP_IN(v0 + (long long)j * sv, nvec_all, p.status)) {
          } else if (valid == EPT) {
            out[(size_t)j * sv] = ov;
            if (NORM) {
#pragma unroll
              for (int e = 0; e < EPT; ++e) part += F::abs2(oe[e]);
            }
          } else {
            E* os = reinterpret_cast<E*>(out + (size_t)j * sv);
            for (int e = 0; e < valid; ++e) {
              os[e] = oe[e];
              if (NORM) part += F::abs2(oe[e]);
            }
          }
        }
      }
      if (NORM) acc = ff_add(acc, FF{part, 0.f});
    }
  }
  return acc;
}


// The same segment with the turn's P new inputs copied to shared memory one turn
// ahead (cp.async, 16 bytes per input): the copies of turn b + 1 are in flight while
// turn b is computed, and they hold no registers, so the kernel keeps more warps
// resident than the register form above.  `slots` is the block's [2][P][blockDim]
// array of 16-byte slots; a thread uses only its own.  The odd images past the
// line's ends are copied from their mirror positions and negated when read.
template <class R, bool CPLX, int AXIS, bool NORM, int W>
__device__ __forceinline__ FF band_line_thread_cp(const LineArgs<typename Field<R, CPLX>::E>& p,
                                                      long long t, float4* slots) {
  using F = Field<R, CPLX>;
  using E = typename F::E;
  constexpr int EPT = 16 / (int)sizeof(E);
  constexpr int P = 2 * W + 1;
  const int nx = p.nx, n = p.n, Ls = p.Ls;
  const int nvec = (nx + EPT - 1) / EPT;
  const int nother = AXIS == 1 ? p.nz : p.ny;
  const int nseg = (n + Ls - 1) / Ls;
  const E* wt = p.wt;
  const int bt = blockDim.x, tid = threadIdx.x;
  FF acc = FF{0.f, 0.f};
  if (t < (long long)nvec * nother * nseg) {
    // t < nvec * nother * nseg <= 1024 * 2048 * 293 < 2^31 (extents <= 2048, segments
    // of at least 2W + 1 >= 7 points): 32-bit division, not 64-bit
    const unsigned int tu = (unsigned int)t;
    const int xv = (int)(tu % (unsigned int)nvec);
    const unsigned int rest = tu / (unsigned int)nvec;
    const int o = (int)(rest % (unsigned int)nother), sg = (int)(rest / (unsigned int)nother);
    const size_t pitch = (size_t)p.pitch;
    const size_t base = (AXIS == 1 ? (size_t)o * p.ny * pitch : (size_t)o * pitch) + (size_t)xv * EPT;
    const float4* in = reinterpret_cast<const float4*>(p.psi + base);
    float4* out = reinterpret_cast<float4*>(p.out + base);
    const size_t sv = (AXIS == 1 ? pitch : pitch * p.ny) * sizeof(E) / 16;   // line stride in vectors
    const int valid = min(EPT, nx - xv * EPT);   // elements of this vector inside the field
    const int j0 = sg * Ls, j1 = min(n, j0 + Ls);
    const bool interior = j0 >= W && j0 + Ls + W <= n;
    // input j of the odd extension about the ghosts -1 and n
    // 16-byte vectors of the field, and this line's first one (bounds checks)
    const long long nvec_all = (long long)p.nz * p.ny * (long long)pitch / EPT, v0 = (long long)(base / EPT);
    // the segment; INTERIOR (no ghost or image within reach, and the vector wholly
    // inside the field: the common case) is a compile-time constant in each of the two
    // instantiations
    auto run = [&](auto interior_c) {
      constexpr bool INTERIOR = decltype(interior_c)::value;
      auto ld = [&](int j) -> float4 {
        if (INTERIOR || (j >= 0 && j < n))
          return GP_IN(v0 + (long long)j * sv, nvec_all, p.status) ? in[(size_t)j * sv]
                                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        if (j == -1 || j == n) return make_float4(0.f, 0.f, 0.f, 0.f);
        const int m = j < 0 ? -2 - j : 2 * n - j;
        const float4 v = GP_IN(v0 + (long long)m * sv, nvec_all, p.status) ? in[(size_t)m * sv]
                                                                           : make_float4(0.f, 0.f, 0.f, 0.f);
        return make_float4(-v.x, -v.y, -v.z, -v.w);
      };
      // copy of turn b's inputs j = b + u + W (u < P) into slot set h
      auto issue = [&](int b, int h) {
#pragma unroll
        for (int u = 0; u < P; ++u) {
          const int j = b + u + W;
          int src = j;
          bool ok = true;
          if (!INTERIOR) {
            ok = b + u < j1 && j != -1 && j != n;
            src = j < 0 ? -2 - j : (j > n ? 2 * n - j : j);
            if (!ok) src = 0;
          }
          if (!GP_IN(v0 + (long long)src * sv, nvec_all, p.status)) ok = false, src = 0;
          cp_async16_zfill(slots + (size_t)(h * P + u) * bt + tid, in + (size_t)src * sv, ok);
        }
      };
      float4 ring[P];
#pragma unroll
      for (int m = 0; m < 2 * W; ++m) ring[m] = ld(j0 - W + m);
      issue(j0, 0);
      cp_async_commit();
      int h = 0;
      for (int b = j0; b < j1; b += P, h ^= 1) {
        if (b + P < j1) issue(b + P, h ^ 1);
        cp_async_commit();
        cp_async_wait<1>();   // turn b's copies have landed
        float part = 0.f;
#pragma unroll
        for (int u = 0; u < P; ++u) {
          const int j = b + u;
          if (INTERIOR || j < j1) {
            float4 v = slots[(size_t)(h * P + u) * bt + tid];
            if (!INTERIOR) {
              const int jj = j + W;
              if (jj < -1 || jj > n) v = make_float4(-v.x, -v.y, -v.z, -v.w);
            }
            ring[(u + 2 * W) % P] = v;
            const E* c = reinterpret_cast<const E*>(&ring[(u + W) % P]);
            float4 ov;
            E* oe = reinterpret_cast<E*>(&ov);
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
              E a = F::mul(wt[W], c[e]);
#pragma unroll
              for (int k = 1; k <= W; ++k) {
                const E* lo = reinterpret_cast<const E*>(&ring[(u + W - k) % P]);
                const E* hi = reinterpret_cast<const E*>(&ring[(u + W + k) % P]);
                a = F::chain(wt[W + k], F::add(lo[e], hi[e]), a);
              }
              oe[e] = F::add(c[e], a);
            }
            if (!GP_IN(v0 + (long long)j * sv, nvec_all, p.status)) {
            } else if (INTERIOR || valid == EPT) {
              out[(size_t)j * sv] = ov;
              if (NORM) {
#pragma unroll
                for (int e = 0; e < EPT; ++e) part += F::abs2(oe[e]);
              }
            } else {
              E* os = reinterpret_cast<E*>(out + (size_t)j * sv);
              for (int e = 0; e < valid; ++e) {
                os[e] = oe[e];
                if (NORM) part += F::abs2(oe[e]);
              }
            }
          }
        }
        if (NORM) acc = ff_add(acc, FF{part, 0.f});
      }

    };
    if (interior && valid == EPT) run(std::true_type{});
    else run(std::false_type{});
    cp_async_wait<0>();
  }
  return acc;
}

template <class R, bool CPLX, int AXIS, bool NORM, int W, bool CP>
__global__ void __launch_bounds__(128) k_sweep_band_line(const __grid_constant__ SweepParams p) {
  pdl_begin();
  // the factor's dither (FP32, imaginary time): the step's x sweep has read the counter
  if (AXIS == 1 && p.step_ctr && blockIdx.x == 0 && threadIdx.x == 0) *p.step_ctr += 1;
  using E = typename Field<R, CPLX>::E;
  LineArgs<E> a;
  a.psi = static_cast<const E*>(p.psi);
  a.out = static_cast<E*>(p.out);
  a.wt = reinterpret_cast<const E*>(p.band_wt);
  a.nx = p.nx;
  a.ny = p.ny;
  a.nz = p.nz;
  a.n = p.n;
  a.pitch = p.pitch;
  a.Ls = p.band_seg;
  a.status = p.status;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  FF acc;
  if constexpr (CP) {
    extern __shared__ __align__(16) float4 band_slots[];
    acc = band_line_thread_cp<R, CPLX, AXIS, NORM, W>(a, t, band_slots);
  } else {
    acc = band_line_thread<R, CPLX, AXIS, NORM, W>(a, t);
  }
  if (NORM) {
    // the block's per-warp sums in shared memory: the cp.async slots when the kernel
    // has them (idle now: every thread has waited for its copies and the barrier
    // orders their last reads), so that the kernel keeps no static shared memory and
    // five 45 KB blocks fit an SM
    FF* wsh;
    if constexpr (CP) {
      extern __shared__ __align__(16) float4 band_slots[];
      __syncthreads();
      wsh = reinterpret_cast<FF*>(band_slots);
    } else {
      __shared__ FF wsh_static[kMaxBlockWarps + 1];
      wsh = wsh_static;
    }
    if (p.norm_defer) {
      // the partial only; the next reader of the factor sums the partials
      FF* wdef = wsh;
      FF b = acc;
      for (int o = 16; o > 0; o >>= 1) b = ff_add(b, ff_shfl_down(b, o));
      if ((threadIdx.x & 31) == 0) wdef[threadIdx.x >> 5] = b;
      __syncthreads();
      if (threadIdx.x == 0) {
        FF s = wdef[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = ff_add(s, wdef[w]);
        for (int c = 0; c < p.norm_copies; ++c)
          reinterpret_cast<FF*>(p.partials)[(size_t)c * gridDim.x + blockIdx.x] = s;
        if (blockIdx.x == 0) *p.scale_state = 1;
      }
    } else {
      norm_finish_ff(acc, reinterpret_cast<FF*>(p.partials), p.counter, gridDim.x, blockIdx.x,
                     p.scale_out, p.status, p.dV, p.counter + kNormGroupBase, kNormGroups, wsh);
    }
  }
}

// Batched y / z sweep: block b of the launch is block blk of nblk of one slot; the
// z sweep's norm is reduced per slot (its own partials, counter and factor).
template <class R, bool CPLX, int AXIS, bool NORM, int W>
__global__ void __launch_bounds__(128) k_batch_band_line(const __grid_constant__ BatchArgs b) {
  pdl_begin();
  using E = typename Field<R, CPLX>::E;
  const LineBlock lb = static_cast<const LineBlock*>(b.items)[blockIdx.x];
  const SlotDesc& d = b.slots[lb.slot];
  LineArgs<E> a;
  a.psi = static_cast<const E*>(AXIS == 1 ? d.field : d.staging);
  a.out = static_cast<E*>(AXIS == 1 ? d.staging : d.field);
  a.wt = reinterpret_cast<const E*>(d.wt[AXIS]) + (kBandHalfMax - W);
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.n = AXIS == 1 ? d.ny : d.nz;
  a.pitch = d.pitch;
  a.Ls = d.seg[AXIS];
  a.status = b.status;
  // the next turn's inputs copied to shared memory ahead, as in k_sweep_band_line
  extern __shared__ __align__(16) float4 band_slots[];
  const FF acc = band_line_thread_cp<R, CPLX, AXIS, NORM, W>(a, (long long)lb.blk * blockDim.x + threadIdx.x,
                                                             band_slots);
  if (NORM) {
    __syncthreads();   // the slots are idle now: the norm's per-warp sums go there
    norm_finish_ff(acc, reinterpret_cast<FF*>(d.partials), d.counter, (unsigned int)lb.nblk,
                   (unsigned int)lb.blk, d.scale, b.status, d.dV, nullptr, 1,
                   reinterpret_cast<FF*>(band_slots));
  }
}

// ---------------------------------------------------------------- launchers

template <class R>
cudaError_t launch_sweep_x(const SweepParams& p, bool complex_field, size_t smem,
                           cudaStream_t st) {
  const long long nrows = (long long)p.ny * p.nz;
  const dim3 grid((unsigned int)((nrows + p.lines - 1) / p.lines));
  return complex_field ? launch_pdl(k_sweep_x<R, true>, grid, 32, smem, st, p)
                       : launch_pdl(k_sweep_x<R, false>, grid, 32, smem, st, p);
}

template <class R>
cudaError_t launch_sweep_y(const CUtensorMap& map, const SweepParams& p, bool complex_field,
                           size_t smem, cudaStream_t st) {
  const dim3 grid((unsigned int)p.tiles_x, (unsigned int)p.nz);
  return complex_field ? launch_pdl(k_sweep_y<R, true>, grid, 32, smem, st, map, p)
                       : launch_pdl(k_sweep_y<R, false>, grid, 32, smem, st, map, p);
}

template <class R>
cudaError_t launch_sweep_z(const CUtensorMap& map, const SweepParams& p, bool complex_field,
                           size_t smem, cudaStream_t st) {
  const dim3 grid((unsigned int)p.tiles_x, (unsigned int)p.ny);
  return complex_field ? launch_pdl(k_sweep_z<R, true, false>, grid, 32, smem, st, map, p)
                       : launch_pdl(k_sweep_z<R, false, true>, grid, 32, smem, st, map, p);
}

// FP32 shared-memory-free sweeps; `trunc` is the truncation depth L (3, 5 or 8),
// `seg` the x-sweep segment per lane (8 or 16).
// Launch with programmatic dependent launch allowed: the kernel's blocks may be
// scheduled while the previous kernel of the stream drains; every sweep kernel waits
// (griddepcontrol.wait) for that kernel's completion before touching memory.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int L>
static cudaError_t launch_fast_L(int axis, const SweepParams& p, bool cplx, int grid,
                                 cudaStream_t st) {
  if (axis == 0) {  // streaming x kernel (1-warp blocks)
    const size_t smem = (size_t)4 * 32 * kXS * (cplx ? 8 : 4);
    const unsigned int blocks = (unsigned int)(((long long)p.ny * p.nz + 31) / 32);
    return cplx ? launch_pdl(k_sweep_x_stream<float, true, L>, blocks, 32, smem, st, p)
                : launch_pdl(k_sweep_x_stream<float, false, L>, blocks, 32, smem, st, p);
  }
  if (axis == 1)
    return cplx ? launch_pdl(k_sweep_stream<float, true, 1, false, L>, grid, 128, 0, st, p)
                : launch_pdl(k_sweep_stream<float, false, 1, false, L>, grid, 128, 0, st, p);
  return cplx ? launch_pdl(k_sweep_stream<float, true, 2, false, L>, grid, 128, 0, st, p)
              : launch_pdl(k_sweep_stream<float, false, 2, true, L>, grid, 128, 0, st, p);
}

template <int L>
static int stream_warps_per_sm_L(int axis, bool cplx) {
  int b = 0;
  if (axis == 1) {
    if (cplx) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_stream<float, true, 1, false, L>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_stream<float, false, 1, false, L>, 128, 0);
  } else {
    if (cplx) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_stream<float, true, 2, false, L>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_stream<float, false, 2, true, L>, 128, 0);
  }
  return 4 * std::max(b, 1);
}

int stream_warps_per_sm(int axis, bool complex_field, int trunc) {
  switch (trunc) {
    case 3: return stream_warps_per_sm_L<3>(axis, complex_field);
    case 5: return stream_warps_per_sm_L<5>(axis, complex_field);
    case 8: return stream_warps_per_sm_L<8>(axis, complex_field);
    default: return 4;
  }
}

template <int W> static auto band_kernel(bool cplx, bool grouped) {
  if (grouped) return cplx ? k_sweep_x_band<float, true, W, true> : k_sweep_x_band<float, false, W, true>;
  return cplx ? k_sweep_x_band<float, true, W, false> : k_sweep_x_band<float, false, W, false>;
}

static void (*band_kernel_for(int w, bool cplx, bool grouped))(SweepParams) {
  switch (w) {
    case 3: return band_kernel<3>(cplx, grouped);
    case 5: return band_kernel<5>(cplx, grouped);
    case 8: return band_kernel<8>(cplx, grouped);
    default: return nullptr;
  }
}

size_t x_band_smem(const SweepParams& p, bool complex_field) {
  return 128 * kBandWarps + (size_t)kBandWarps * p.band_stages * p.band_group *
                                (p.pitch + 2 * kBandPad) * (complex_field ? 8 : 4);
}

int x_band_group(int nx, int ept, int stages, size_t slot_bytes, size_t warp_budget) {
  // rows per group: cost per element of a group of G rows in warp instructions, from
  // the measured split of the kernel (pointwise and dot products per 32 vectors, odd
  // images per 32 of the 15 tasks per row, fixed work per group)
  const int nvec = (nx + ept - 1) / ept;
  int best = 1;
  double best_cost = 1e300;
  for (int g = 1; g <= 8; ++g) {
    if (g > 1 && (size_t)stages * g * slot_bytes > warp_budget) break;
    const double cost = (((g * nvec + 31) / 32) * 112.0 + ((15 * g + 31) / 32) * 15.0 + 40.0) /
                        ((double)g * nx);
    if (cost < best_cost * 0.98) {
      best_cost = cost;
      best = g;
    }
  }
  return best;
}

cudaError_t x_band_prepare(int w, bool complex_field, bool grouped, size_t smem, int* blocks_per_sm) {
  void (*k)(SweepParams) = band_kernel_for(w, complex_field, grouped);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * kBandWarps, smem);
}

static void (*x_reg_kernel_for(int w, bool cplx))(SweepParams) {
  switch (w) {
    case 3: return cplx ? k_sweep_x_reg<true, 3> : k_sweep_x_reg<false, 3>;
    case 5: return cplx ? k_sweep_x_reg<true, 5> : k_sweep_x_reg<false, 5>;
    default: return nullptr;
  }
}

bool x_reg_fits(int nx, int w) { return nx % 8 == 0 && nx <= 256 && (w == 3 || w == 5); }

cudaError_t x_reg_prepare(int w, bool complex_field, int* blocks_per_sm) {
  void (*k)(SweepParams) = x_reg_kernel_for(w, complex_field);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * kXRegWarps, 0);
}

cudaError_t launch_sweep_x_reg(const SweepParams& p, bool complex_field, int grid, cudaStream_t st) {
  void (*k)(SweepParams) = x_reg_kernel_for(p.band_w, complex_field);
  if (!k) return cudaErrorInvalidValue;
  return launch_pdl(k, grid, 32 * kXRegWarps, 0, st, p);
}

cudaError_t launch_sweep_x_band(const SweepParams& p, bool complex_field, int grid,
                                cudaStream_t st) {
  void (*k)(SweepParams) = band_kernel_for(p.band_w, complex_field, p.band_group > 1);
  if (!k) return cudaErrorInvalidValue;
  return launch_pdl(k, grid, 32 * kBandWarps, x_band_smem(p, complex_field), st, p);
}

// shared memory of a banded y / z block: 128 threads x two turns of 2W+1 16-byte slots
static size_t band_line_smem(int W, bool cp) { return cp ? (size_t)128 * 2 * (2 * W + 1) * 16 : 0; }

using SweepKernel = void (*)(SweepParams);
template <int W, bool CP> static SweepKernel band_line_kernel(int axis, bool cplx) {
  if (axis == 1)
    return cplx ? k_sweep_band_line<float, true, 1, false, W, CP> : k_sweep_band_line<float, false, 1, false, W, CP>;
  return cplx ? k_sweep_band_line<float, true, 2, false, W, CP> : k_sweep_band_line<float, false, 2, true, W, CP>;
}

template <int W>
static cudaError_t launch_band_line_W(int axis, const SweepParams& p, bool cplx, int grid,
                                     cudaStream_t st) {
  const bool cp = p.band_cp != 0;
  void (*k)(SweepParams) = cp ? band_line_kernel<W, true>(axis, cplx) : band_line_kernel<W, false>(axis, cplx);
  return launch_pdl(k, grid, 128, band_line_smem(W, cp), st, p);
}

template <int W> static int band_line_blocks_per_sm_W(int axis, bool cplx, bool cp) {
  void (*k)(SweepParams) = cp ? band_line_kernel<W, true>(axis, cplx) : band_line_kernel<W, false>(axis, cplx);
  const size_t smem = band_line_smem(W, cp);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, 128, smem);
  return b;
}

int band_line_blocks_per_sm(int axis, bool complex_field, int w, bool cp) {
  switch (w) {
    case 3: return band_line_blocks_per_sm_W<3>(axis, complex_field, cp);
    case 5: return band_line_blocks_per_sm_W<5>(axis, complex_field, cp);
    case 8: return band_line_blocks_per_sm_W<8>(axis, complex_field, cp);
    default: return 0;
  }
}

cudaError_t launch_sweep_band_line(int axis, const SweepParams& p, bool complex_field, int grid,
                                   cudaStream_t st) {
  switch (p.band_w) {
    case 3: return launch_band_line_W<3>(axis, p, complex_field, grid, st);
    case 5: return launch_band_line_W<5>(axis, p, complex_field, grid, st);
    case 8: return launch_band_line_W<8>(axis, p, complex_field, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t batch_x_smem(int stages, int group_max, int slot_elems, bool complex_field) {
  return 128 * kBatchXWarps +
         (size_t)kBatchXWarps * stages * group_max * slot_elems * (complex_field ? 8 : 4);
}

// the batched y / z kernels' turn slots (above 48 KB at W = 8), every mode and axis
template <int W> static cudaError_t batch_yz_prepare() {
  void (*const yz[4])(BatchArgs) = {k_batch_band_line<float, false, 1, false, W>,
                                    k_batch_band_line<float, false, 2, true, W>,
                                    k_batch_band_line<float, true, 1, false, W>,
                                    k_batch_band_line<float, true, 2, false, W>};
  for (auto k : yz) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)band_line_smem(W, true));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int W> static cudaError_t batch_prepare_W(bool cplx, size_t x_smem, int* bps) {
  void (*k)(BatchArgs) = cplx ? k_batch_x_band<float, true, W> : k_batch_x_band<float, false, W>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)x_smem);
  if (e != cudaSuccess) return e;
  if ((e = batch_yz_prepare<3>()) != cudaSuccess || (e = batch_yz_prepare<5>()) != cudaSuccess ||
      (e = batch_yz_prepare<8>()) != cudaSuccess)
    return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, 32 * kBatchXWarps, x_smem);
}

cudaError_t batch_prepare(int w, bool complex_field, size_t x_smem, int* x_blocks_per_sm) {
  switch (w) {
    case 3: return batch_prepare_W<3>(complex_field, x_smem, x_blocks_per_sm);
    case 5: return batch_prepare_W<5>(complex_field, x_smem, x_blocks_per_sm);
    case 8: return batch_prepare_W<8>(complex_field, x_smem, x_blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

template <int W>
static cudaError_t launch_batch_W(int axis, const BatchArgs& b, bool cplx, int grid, size_t smem,
                                  cudaStream_t st) {
  if (axis == 0 && b.x_reg) {
    if constexpr (W <= 7)
      return cplx ? launch_pdl(k_batch_x_reg<true, W>, grid, 32 * kXRegWarps, 0, st, b)
                  : launch_pdl(k_batch_x_reg<false, W>, grid, 32 * kXRegWarps, 0, st, b);
    return cudaErrorInvalidValue;
  }
  if (axis == 0)
    return cplx ? launch_pdl(k_batch_x_band<float, true, W>, grid, 32 * kBatchXWarps, smem, st, b)
                : launch_pdl(k_batch_x_band<float, false, W>, grid, 32 * kBatchXWarps, smem, st, b);
  const size_t ysmem = band_line_smem(W, true);
  if (axis == 1)
    return cplx ? launch_pdl(k_batch_band_line<float, true, 1, false, W>, grid, 128, ysmem, st, b)
                : launch_pdl(k_batch_band_line<float, false, 1, false, W>, grid, 128, ysmem, st, b);
  return cplx ? launch_pdl(k_batch_band_line<float, true, 2, false, W>, grid, 128, ysmem, st, b)
              : launch_pdl(k_batch_band_line<float, false, 2, true, W>, grid, 128, ysmem, st, b);
}

bool batch_x_reg_fits(int nx, int w, bool complex_field) {
  const int epl = complex_field ? 8 : 16;
  return nx % epl == 0 && nx <= 32 * epl && (w == 3 || w == 5);
}

cudaError_t batch_x_reg_prepare(int w, bool complex_field, int* blocks_per_sm) {
  void (*k)(BatchArgs) = nullptr;
  if (w == 3) k = complex_field ? k_batch_x_reg<true, 3> : k_batch_x_reg<false, 3>;
  if (w == 5) k = complex_field ? k_batch_x_reg<true, 5> : k_batch_x_reg<false, 5>;
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * kXRegWarps, 0);
}

cudaError_t launch_batch_sweep(int axis, int w, const BatchArgs& b, bool complex_field, int grid,
                               size_t smem, cudaStream_t st) {
  switch (w) {
    case 3: return launch_batch_W<3>(axis, b, complex_field, grid, smem, st);
    case 5: return launch_batch_W<5>(axis, b, complex_field, grid, smem, st);
    case 8: return launch_batch_W<8>(axis, b, complex_field, grid, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sweep_fast(int axis, const SweepParams& p, bool complex_field, int grid,
                              cudaStream_t st) {
  switch (p.trunc) {
    case 3: return launch_fast_L<3>(axis, p, complex_field, grid, st);
    case 5: return launch_fast_L<5>(axis, p, complex_field, grid, st);
    case 8: return launch_fast_L<8>(axis, p, complex_field, grid, st);
    default: return cudaErrorInvalidValue;
  }
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
