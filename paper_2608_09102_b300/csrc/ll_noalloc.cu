// ll_residual_noalloc: the residual of a candidate solution for callers that
// cannot allocate device memory (see include/ll_mg.h).  Its reduction scratch
// is a fixed file-scope device array instead of a cudaMalloc'd buffer.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "../../include/ll_mg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr long kCellsPerBlock = (long)kThreads * kCellsPerThread;  // 4096
constexpr int kMaxBlocks = 2048;                                  // => at most 8,388,608 cells
constexpr int kMaxDevices = 64;

// Two partial sums per block (|r|^2 and |b|^2): 32 KB, kept by every device
// that loads the library until the process exits.  Each call overwrites the
// slots it uses before reading them, so nothing needs clearing; calls that
// overlap on the GPU share this array and race.
static __device__ __align__(256) double g_partial[2 * kMaxBlocks];

// Device address of g_partial per device, looked up once per device.  In host
// code the name g_partial is only a host-side stand-in for the symbol, so
// kernels are always given the address obtained here.
double* g_partial_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LL_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LL_ELIMIT;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partial) != cudaSuccess || !p) return LL_ECUDA;
    g_partial_addr[dev] = (double*)p;
  }
  *out = g_partial_addr[dev];
  return LL_OK;
}

// r = b - A x per cell on the natural grid, with C(m)/h^2 formed on the fly;
// per-block partial sums of |r|^2 and |b|^2 go to partial[2*block + q].
__global__ void k_residual_partial(int nx, int ny, int nz, const double* __restrict__ m, double alpha,
                                   double inv_dt, double ih2, const double* __restrict__ b,
                                   const double* __restrict__ x, double* __restrict__ r,
                                   double* __restrict__ partial) {
  long n = (long)nx * ny * nz;
  long k0 = blockIdx.x * kCellsPerBlock;
  long k1 = k0 + kCellsPerBlock < n ? k0 + kCellsPerBlock : n;
  double rr = 0.0, bb = 0.0;
  for (long k = k0 + threadIdx.x; k < k1; k += kThreads) {
    int i = (int)(k % nx);
    long t = k / nx;
    int j = (int)(t % ny), l = (int)(t / ny);
    long nxy = (long)nx * ny;
    // face neighbours present (Neumann: missing ones are left out), tested
    // in place rather than gathered into an index array, which would sit in
    // local memory and serialise the loads
    bool zm = l > 0, ym = j > 0, xm = i > 0, xp = i < nx - 1, yp = j < ny - 1, zp = l < nz - 1;
    int d = zm + ym + xm + xp + yp + zp;
    double lap[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double* xc = x + c * n + k;
      double s = 0.0;
      if (zm) s += xc[-nxy];
      if (ym) s += xc[-nx];
      if (xm) s += xc[-1];
      if (xp) s += xc[1];
      if (yp) s += xc[nx];
      if (zp) s += xc[nxy];
      lap[c] = (s - d * xc[0]) * ih2;  // (Delta_h x)_k
    }
    double m1 = m[k], m2 = m[n + k], m3 = m[2 * n + k];
    double mm = m1 * m1 + m2 * m2 + m3 * m3;
    double md = m1 * lap[0] + m2 * lap[1] + m3 * lap[2];
    // C(m) v = m x v + alpha (m (m.v) - |m|^2 v)
    double cv[3] = {m2 * lap[2] - m3 * lap[1] + alpha * (m1 * md - mm * lap[0]),
                    m3 * lap[0] - m1 * lap[2] + alpha * (m2 * md - mm * lap[1]),
                    m1 * lap[1] - m2 * lap[0] + alpha * (m3 * md - mm * lap[2])};
    for (int c = 0; c < 3; ++c) {
      double bv = b[c * n + k];
      double v = bv - (x[c * n + k] * inv_dt + cv[c]);
      if (r) r[c * n + k] = v;
      rr += v * v;
      bb += bv * bv;
    }
  }
  __shared__ double s0[kThreads], s1[kThreads];
  s0[threadIdx.x] = rr;
  s1[threadIdx.x] = bb;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0[0];
    partial[2 * blockIdx.x + 1] = s1[0];
  }
}

// out[q] = sum over the blocks of partial[2*block + q], in a fixed order
__global__ void k_residual_finish(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  __shared__ double s0[kThreads], s1[kThreads];
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kThreads) {
    a += partial[2 * i];
    c += partial[2 * i + 1];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = c;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
  }
}

}  // namespace

extern "C" int ll_residual_noalloc(const double* m_tilde, double alpha, double dt, double h, ll_grid grid,
                                   const double* rhs, const double* x, double* r, double* norms2,
                                   void* cuda_stream) {
  if (!m_tilde || !rhs || !x || !norms2) return LL_EINVAL;
  if (!(dt > 0) || !(h > 0) || !(alpha >= 0) || !isfinite(dt) || !isfinite(h) || !isfinite(alpha))
    return LL_EINVAL;
  if (grid.nx < 1 || grid.ny < 1 || grid.nz < 1) return LL_EINVAL;
  long n = (long)grid.nx * grid.ny * grid.nz;
  if (n > kCellsPerBlock * kMaxBlocks) return LL_ELIMIT;  // beyond the fixed scratch
  double* partial = nullptr;
  int st = scratch_address(&partial);
  if (st != LL_OK) return st;
  int nblocks = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_residual_partial<<<nblocks, kThreads, 0, s>>>(grid.nx, grid.ny, grid.nz, m_tilde, alpha, 1.0 / dt,
                                                  1.0 / (h * h), rhs, x, r, partial);
  if (cudaGetLastError() != cudaSuccess) return LL_ECUDA;
  k_residual_finish<<<1, kThreads, 0, s>>>(partial, nblocks, norms2);
  if (cudaGetLastError() != cudaSuccess) return LL_ECUDA;
  return LL_OK;
}
