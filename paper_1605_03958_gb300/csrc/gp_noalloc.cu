// gp_noalloc.cu -- gp_observables_noalloc: the observables reduction over a field that
// lives in the caller's device memory, with no device allocation at all.
//
// Who needs this: callers that must not call cudaMalloc.  cudaMalloc (and the solver's
// gp_create) implicitly synchronises the device, which stalls every other stream of a
// latency-sensitive loop; it can fail although memory is free when another allocator
// (PyTorch's caching allocator, a framework's memory pool) holds that memory; and some
// host programs that load this library as a plugin forbid device allocation from
// inside their callbacks.  Such callers already own the field and an output buffer;
// this entry point needs nothing else.
//
// The reduction's scratch (one partial sum per block and accumulator, plus the
// last-block ticket counter) lives in the file-scope array below, which every GPU that
// loads this library holds until the process exits.  All calls share it: a call clears
// the counter before its kernel runs and overwrites every partial it reads, but two
// calls whose kernels overlap on the GPU (different streams, no ordering between them)
// race on the array and produce wrong results.  Order such calls on one stream.
//
// The paper has no counterpart: this is an operational variant of gp_observables.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/gp.h"
#include "gp_device.cuh"

namespace {

// Maximum scratch: 64 KiB.  Layout: [0, 256) ticket counter, [256, ...) partials.
constexpr size_t kScratchBytes = 64 * 1024;
constexpr size_t kPartialsOffset = 256;
constexpr int kBlocks = gpk::kReduceBlocks;   // same launch shape as gp_observables
constexpr int kThreads = gpk::kReduceThreads;
constexpr int kAcc = gpk::kObsAcc;
static_assert(kPartialsOffset + sizeof(double) * kBlocks * kAcc <= kScratchBytes,
              "reduction partials must fit the static scratch");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, resolved once per device (with that device current).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    gpk::set_thread_error((std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    return GP_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    gpk::set_thread_error("device ordinal beyond the supported range of 64");
    return GP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      gpk::set_thread_error((std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
      return GP_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return GP_OK;
}

template <class R, bool CPLX> struct Load;
template <class R> struct Load<R, false> {
  static __device__ __forceinline__ double2 at(const void* psi, size_t idx) {
    return make_double2((double)static_cast<const R*>(psi)[idx], 0.0);
  }
};
template <class R> struct Load<R, true> {
  static __device__ __forceinline__ double2 at(const void* psi, size_t idx) {
    const typename gpk::Cplx<R>::T v = static_cast<const typename gpk::Cplx<R>::T*>(psi)[idx];
    return make_double2((double)v.x, (double)v.y);
  }
};

__device__ __forceinline__ double abs2(double2 v) { return fma(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ double abs2_diff(double2 a, double2 b) {
  const double x = a.x - b.x, y = a.y - b.y;
  return fma(x, x, y * y);
}

struct Args {
  const void* psi;
  int nx, ny, nz;
  long long pitch;
  double hx, hy, hz;
  double wx, wy, wz;   // trap frequencies gamma, nu, lambda
  double g;
  double* out;         // 10 doubles, caller's device memory
  unsigned int* counter;
  double* partials;
};

// Same accumulators, order and launch shape as the solver's observables pass; the
// trap potential and x^2 come from the grid coordinates instead of tables.
template <class R, bool CPLX>
__global__ void __launch_bounds__(kThreads) k_observables_noalloc(const Args a) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t P = (size_t)a.pitch, plane = P * ny;
  double acc[kAcc];
#pragma unroll
  for (int c = 0; c < kAcc; ++c) acc[c] = 0.0;
  const long long nrows = (long long)ny * nz;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const double y = (j - 0.5 * (ny - 1)) * a.hy, z = (k - 0.5 * (nz - 1)) * a.hz;
    const double y2 = y * y, z2 = z * z;
    const double vyz = 0.5 * a.wy * a.wy * y2 + 0.5 * a.wz * a.wz * z2;
    const size_t base = (size_t)r * P;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double x = (i - 0.5 * (nx - 1)) * a.hx;
      const size_t idx = base + i;
      const double2 v = Load<R, CPLX>::at(a.psi, idx);
      const double d = abs2(v);
      const double2 z0 = make_double2(0.0, 0.0);
      const double2 wxn = (i + 1 < nx) ? Load<R, CPLX>::at(a.psi, idx + 1) : z0;
      const double2 wyn = (j + 1 < ny) ? Load<R, CPLX>::at(a.psi, idx + P) : z0;
      const double2 wzn = (k + 1 < nz) ? Load<R, CPLX>::at(a.psi, idx + plane) : z0;
      acc[0] += d;
      acc[1] += (0.5 * a.wx * a.wx * x * x + vyz) * d;
      acc[2] += d * d;
      acc[3] += abs2_diff(wxn, v) + (i == 0 ? d : 0.0);
      acc[4] += abs2_diff(wyn, v) + (j == 0 ? d : 0.0);
      acc[5] += abs2_diff(wzn, v) + (k == 0 ? d : 0.0);
      acc[6] += x * x * d;
      acc[7] += y2 * d;
      acc[8] += z2 * d;
    }
  }

  // fixed-order block sums -> partials in the static scratch; last block finishes
  __shared__ double warp_part[kThreads / 32][kAcc];
  __shared__ double tot[kAcc];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kAcc; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) warp_part[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kAcc) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += warp_part[w][threadIdx.x];
    a.partials[(size_t)blockIdx.x * kAcc + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < kAcc) {
    double s = 0.0, comp = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) {
      const double x = __ldcg(a.partials + (size_t)b * kAcc + threadIdx.x);
      const double u = s + x;
      comp += (fabs(s) >= fabs(x)) ? (s - u) + x : (x - u) + s;
      s = u;
    }
    tot[threadIdx.x] = s + comp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *a.counter = 0u;
    // nz = 1 is a 2D field in the xy plane: cell area hx hy and no z kinetic term
    // (every point has k = 0 there, so z = 0 and V has no z part already)
    const bool two_d = nz == 1;
    const double dV = a.hx * a.hy * (two_d ? 1.0 : a.hz);
    const double norm = tot[0] * dV;
    const double epot = tot[1] * dV;
    const double eint = 0.5 * a.g * tot[2] * dV;
    const double ekin = 0.5 * dV *
                        (tot[3] / (a.hx * a.hx) + tot[4] / (a.hy * a.hy) +
                         (two_d ? 0.0 : tot[5] / (a.hz * a.hz)));
    const double x2 = tot[6] * dV / norm, y2 = tot[7] * dV / norm, z2 = tot[8] * dV / norm;
    double* o = a.out;
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

bool finite_pos(double v) { return v > 0.0 && v < 1e300; }

}  // namespace

extern "C" int gp_observables_noalloc(const void* psi, int nx, int ny, int nz, long long pitch,
                                      int prec, int is_complex, double dx, double dy, double dz,
                                      double gamma, double nu, double lambda, double g,
                                      double* out, void* stream) {
  if (!psi || !out) {
    gpk::set_thread_error("psi and out must be device pointers");
    return GP_ERR_ARG;
  }
  // the extents gp_create accepts: 3..2048 per axis, or nz = 1 for a 2D field
  if (nx < 3 || ny < 3 || (nz < 3 && nz != 1) || nx > gpk::kMaxExtent ||
      ny > gpk::kMaxExtent || nz > gpk::kMaxExtent) {
    gpk::set_thread_error(
        "grid extents must be within 3..2048 (nz = 1: a 2D field), the limit of this entry point");
    return GP_ERR_ARG;
  }
  if (pitch < nx) {
    gpk::set_thread_error("pitch must be >= nx");
    return GP_ERR_ARG;
  }
  if (prec != GP_F64 && prec != GP_F32) {
    gpk::set_thread_error("prec must be GP_F64 or GP_F32");
    return GP_ERR_ARG;
  }
  if (is_complex != 0 && is_complex != 1) {
    gpk::set_thread_error("is_complex must be 0 or 1");
    return GP_ERR_ARG;
  }
  if (nz == 1) dz = lambda = 1.0;   // unused by a 2D field
  if (!finite_pos(dx) || !finite_pos(dy) || !finite_pos(dz) || !finite_pos(gamma) ||
      !finite_pos(nu) || !finite_pos(lambda) || !(g == g)) {
    gpk::set_thread_error("spacings and trap ratios must be finite and > 0, g finite");
    return GP_ERR_ARG;
  }
  unsigned char* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != GP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Args a{psi, nx, ny, nz, pitch, dx, dy, dz, gamma, nu, lambda, g, out,
         reinterpret_cast<unsigned int*>(scratch),
         reinterpret_cast<double*>(scratch + kPartialsOffset)};
  // the ticket counter must start at zero; everything else is overwritten
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    gpk::set_thread_error((std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)).c_str());
    return GP_ERR_CUDA;
  }
  if (prec == GP_F64) {
    if (is_complex) k_observables_noalloc<double, true><<<kBlocks, kThreads, 0, st>>>(a);
    else k_observables_noalloc<double, false><<<kBlocks, kThreads, 0, st>>>(a);
  } else {
    if (is_complex) k_observables_noalloc<float, true><<<kBlocks, kThreads, 0, st>>>(a);
    else k_observables_noalloc<float, false><<<kBlocks, kThreads, 0, st>>>(a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    gpk::set_thread_error((std::string("kernel launch: ") + cudaGetErrorString(e)).c_str());
    return GP_ERR_CUDA;
  }
  return GP_OK;
}

