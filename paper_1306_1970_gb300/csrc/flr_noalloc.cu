// flr_solve_noalloc: the MM solve without any device allocation.
//
// For callers that cannot call cudaMalloc: for example code running inside
// a framework whose caching allocator has already reserved the device's
// memory (a fresh cudaMalloc then fails or fragments that pool), or a
// serving loop that must never take the driver's allocation path, which can
// synchronize the whole device.  Everything the solve needs beyond the
// caller's inputs and outputs lives in one file-scope device array
// (flr_noalloc_scratch) that every GPU loading this library holds until the
// process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and caches
// it.  That first call should therefore come before any stream capture.
// All calls share the array and it keeps the previous call's contents: the
// parts that must start at zero are cleared on every call, and calls whose
// work overlaps on the GPU (other streams, other threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/flr.h"
#include "flr_solve.cuh"

using namespace flr;

namespace {

static __device__ __align__(256) unsigned char flr_noalloc_scratch[FLR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int kMaxGridNA = 512;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Address of the scratch array on device `dev` (looked up once per device).
flr_status scratch_on(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return FLR_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, flr_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      (void)cudaGetLastError();
      return FLR_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return FLR_OK;
}

template <typename TX> __device__ __forceinline__ double widen_na(TX v);
template <> __device__ __forceinline__ double widen_na<double>(double v) { return v; }
template <> __device__ __forceinline__ double widen_na<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double widen_na<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <> __device__ __forceinline__ double widen_na<__half>(__half v) {
  return (double)__half2float(v);
}

// d_j = X_j^T X_j, c_j = X_j^T y (FP64), one warp per column of column-major X
template <typename TX>
__global__ void na_colstats(const TX* __restrict__ Xt, const double* __restrict__ y, long long n,
                            long long p, long long ldn, double* d, double* c) {
  const int lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (j >= p) return;
  const TX* col = Xt + j * ldn;
  double sd = 0.0, sc = 0.0;
  for (long long i = lane; i < n; i += 32) {
    const double v = widen_na<TX>(col[i]);
    sd = fma(v, v, sd);
    sc = fma(v, y[i], sc);
  }
  sd = warp_sum(sd);
  sc = warp_sum(sc);
  if (lane == 0) { d[j] = sd; c[j] = sc; }
}

// out[0] = ||c||_2 (one block)
__global__ void na_norm(const double* __restrict__ c, long long p, double* out) {
  __shared__ double ws[32];
  double s = 0.0;
  for (long long j = threadIdx.x; j < p; j += blockDim.x) s = fma(c[j], c[j], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < blockDim.x / 32 ? ws[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[0] = sqrt(t);
  }
}

size_t esize(int dt) {
  switch (dt) {
    case FLR_F64: return 8;
    case FLR_F32: return 4;
    case FLR_BF16: case FLR_F16: return 2;
    default: return 0;
  }
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

template <typename TX>
flr_status run(const SolveParams& P0, const void* Xt, const double* y, long long n, long long p,
               long long ldn, int G, size_t smem, int sm_count, cudaStream_t st, double* cnorm_dev,
               double* dd, double* cc) {
  na_colstats<TX><<<(unsigned)((p + 7) / 8), 256, 0, st>>>(static_cast<const TX*>(Xt), y, n, p, ldn,
                                                           dd, cc);
  na_norm<<<1, 1024, 0, st>>>(cc, p, cnorm_dev);
  double cn = 0.0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cn, cnorm_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { (void)cudaGetLastError(); return FLR_ECUDA; }
  if (!std::isfinite(cn)) return FLR_ENONFINITE;
  SolveParams P = P0;
  P.cnorm = cn > 0.0 ? cn : 1.0;
  auto kern = mm_solve_kernel<TX, GK_STENCIL>;
  // per-kernel attribute shared with concurrent callers: always the most the
  // device allows next to the kernel's static shared memory
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, (const void*)kern) != cudaSuccess) {
    (void)cudaGetLastError();
    return FLR_ECUDA;
  }
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  if (smem > (size_t)dyn_max) return FLR_ENOTIMPL;
  if (P.ws != 0) {   // slab columns after the TMEM ones resident in shared memory
    P.ws = resident_columns(P.w - P.wt, P.ldn, sizeof(TX), smem, dyn_max);
    if (P.ws > 0) smem = (smem + 15) / 16 * 16 + (size_t)P.ws * (size_t)P.ldn * sizeof(TX);
  }
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
    (void)cudaGetLastError();
    return FLR_ECUDA;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return FLR_ECUDA;
  }
  if (nb < 1 || G > nb * sm_count) return FLR_ENOTIMPL;
  void* args[] = {(void*)&P};
  if (cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(kThreads), args, smem, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return FLR_ECUDA;
  }
  return FLR_OK;
}

}  // namespace

extern "C" flr_status flr_solve_noalloc(const void* Xt, int32_t dtype, int64_t n, int64_t p,
                                        int64_t ldn, const double* y, const flr_graph* E,
                                        double lambda1, double lambda2, double eps, double tol,
                                        const flr_opts* opts, double* beta_out, void* stream,
                                        flr_stats* stats) {
  // ---- arguments
  if (!Xt || !y || !E || !beta_out || n < 1 || p < 1) return FLR_EINVAL;
  const size_t es = esize(dtype);
  if (es == 0 || ldn < n || ((size_t)ldn * es) % 16 != 0) return FLR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(Xt) & 15) != 0) return FLR_EINVAL;
  if (!(lambda1 >= 0.0) || !(lambda2 >= 0.0) || !(eps > 0.0) || !(tol > 0.0)) return FLR_EINVAL;
  if (!std::isfinite(lambda1) || !std::isfinite(lambda2) || !std::isfinite(eps)) return FLR_EINVAL;
  long long q2 = p;
  if (E->kind == FLR_E_LATTICE) {
    if (E->q1 < 1 || E->q2 < 1 || E->q1 * E->q2 != p) return FLR_EINVAL;
    q2 = E->q2;
  } else if (E->kind != FLR_E_CHAIN) {
    return FLR_ENOTIMPL;
  }
  flr_opts o;
  flr_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_mm < 0 || o.max_cg < 0 || o.min_cg < 0 || o.tol_cg < 0.0 || o.wait_cycles < 0 ||
      o.max_refine < 0 || (o.x_smem != 0 && o.x_smem != -1) ||
      !(o.tol_cg_rel >= 0.0))
    return FLR_EINVAL;
  int precond = o.precond;
  if (precond == FLR_PC_AUTO) precond = FLR_PC_TWOLEVEL;
  if (precond != FLR_PC_JACOBI && precond != FLR_PC_TRIDIAG && precond != FLR_PC_PAPER &&
      precond != FLR_PC_TWOLEVEL)
    return FLR_EINVAL;
  const bool two = precond == FLR_PC_TWOLEVEL;
  // the kernel's local tridiagonal solve: TRIDIAG, PAPER, and TWOLEVEL on a chain
  const bool tri = precond == FLR_PC_TRIDIAG || precond == FLR_PC_PAPER || (two && E->kind == FLR_E_CHAIN);

  int dev = 0, sm_count = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return FLR_ECUDA; }
  cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

  // ---- launch shape (same rule as flr_solve)
  const long long per_block = dtype == FLR_F64 ? 8192 : 65536;
  long long G = o.grid > 0 ? o.grid : (n * p + per_block - 1) / per_block;
  G = std::max<long long>(1, std::min<long long>({G, (long long)sm_count, (long long)kMaxGridNA, p}));
  const long long w = (p + G - 1) / G;
  G = (p + w - 1) / w;
  if (w > 8192) return FLR_ENOTIMPL;
  int levels = 0;
  while ((1LL << levels) < w) ++levels;
  const long long wpad = (w + 3) / 4 * 4;
  const int tct = o.x_smem == 0 ? tmem_cells(n, (int)es) : 0;
  const long long trows = tct > 0 ? (n + 127) / 128 * 128 : 0;
  const size_t smem = solve_smem_bytes(ldn, wpad, (int)(16 / es), halo_entries(wpad, q2, p), trows);

  // ---- scratch layout inside the static array
  const size_t vecb = up256(sizeof(double) * (size_t)p);
  size_t off = 0;
  const size_t o_ctl = off;  off += 256;
  const size_t o_part = off; off += up256(sizeof(double) * 2 * kNF * kMaxGridNA);
  const size_t o_cn = off;   off += 256;
  const size_t o_vec = off;  off += 7 * vecb;                       // x z pb0 pb1 c d binv
  const size_t o_two = off;                                          // qcinv qc qci sc0 sc1 uf cmap cid
  if (two) off += 8 * vecb;
  const size_t o_k = off;
  if (tri) off += 2 * up256(sizeof(double) * (size_t)levels * (size_t)p);
  const size_t o_u = off;    off += 2 * up256(sizeof(double) * (size_t)ldn * kUR);
  if (off > (size_t)FLR_NOALLOC_SCRATCH_BYTES) return FLR_ESCRATCH;
  if (smem > (size_t)smem_max) return FLR_ENOTIMPL;

  unsigned char* S = nullptr;
  flr_status s = scratch_on(dev, &S);
  if (s != FLR_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* vec[7];
  for (int i = 0; i < 7; ++i) vec[i] = reinterpret_cast<double*>(S + o_vec + i * vecb);
  double* ub0 = reinterpret_cast<double*>(S + o_u);
  double* ub1 = reinterpret_cast<double*>(S + o_u + up256(sizeof(double) * (size_t)ldn * kUR));

  // ---- what must start at zero (the array keeps the previous call's contents)
  if (cudaMemsetAsync(S + o_ctl, 0, 128, st) != cudaSuccess ||
      cudaMemsetAsync(S + o_ctl + 128, 0xff, 128, st) != cudaSuccess ||
      cudaMemsetAsync(ub0, 0, sizeof(double) * ldn * kUR, st) != cudaSuccess ||
      cudaMemsetAsync(ub1, 0, sizeof(double) * ldn * kUR, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return FLR_ECUDA;
  }

  SolveParams P{};
  P.Xt = Xt; P.n = n; P.p = p; P.ldn = ldn;
  P.y = y; P.c = vec[4]; P.d = vec[5];
  P.q2 = q2;
  P.rowptr = nullptr; P.col = nullptr;
  P.lam1 = lambda1; P.lam2 = lambda2; P.eps = eps; P.tol = tol;
  P.tol_cg = o.tol_cg > 0.0 ? o.tol_cg : tol;
  P.tol_cg_rel = o.tol_cg_rel;
  P.max_mm = o.max_mm; P.max_cg = o.max_cg; P.min_cg = o.min_cg; P.precond = precond;
  P.max_refine = o.max_refine;
  P.ws = o.x_smem == 0 ? 1 : 0;
  P.tct = tct;
  P.wt = tct > 0 ? tct * (4 / (int)es) : 0;
  P.w = w; P.wpad = wpad; P.levels = levels;
  P.beta_init = nullptr;
  P.x = vec[0]; P.z = vec[1]; P.pb0 = vec[2]; P.pb1 = vec[3];
  P.binv = vec[6];
  if (two) {
    double* t[5];
    for (int i = 0; i < 5; ++i) t[i] = reinterpret_cast<double*>(S + o_two + i * vecb);
    P.qcinv = t[0]; P.qc = t[1]; P.qci = t[2]; P.sc0 = t[3]; P.sc1 = t[4];
    P.uf = reinterpret_cast<int*>(S + o_two + 5 * vecb);
    P.cmap = reinterpret_cast<int*>(S + o_two + 6 * vecb);
    P.cid = reinterpret_cast<int*>(S + o_two + 7 * vecb);
    P.ncomp = reinterpret_cast<int*>(S + o_ctl + 96);
  }
  P.K1 = tri ? reinterpret_cast<double*>(S + o_k) : nullptr;
  P.K2 = tri
             ? reinterpret_cast<double*>(S + o_k + up256(sizeof(double) * (size_t)levels * (size_t)p))
             : nullptr;
  P.ub0 = ub0; P.ub1 = ub1;
  P.part = reinterpret_cast<double*>(S + o_part);
  P.bar = reinterpret_cast<unsigned*>(S + o_ctl);
  P.err = reinterpret_cast<int*>(S + o_ctl + 64);
  P.stats = reinterpret_cast<DevStats*>(S + o_ctl + 128);
  P.timeout = o.wait_cycles > 0 ? o.wait_cycles : (1LL << 33);
  P.inject_stall = o.inject_stall;

  const auto t0 = std::chrono::steady_clock::now();
  double* cnorm_dev = reinterpret_cast<double*>(S + o_cn);
  switch (dtype) {
    case FLR_F64: s = run<double>(P, Xt, y, n, p, ldn, (int)G, smem, sm_count, st, cnorm_dev, vec[5], vec[4]); break;
    case FLR_F32: s = run<float>(P, Xt, y, n, p, ldn, (int)G, smem, sm_count, st, cnorm_dev, vec[5], vec[4]); break;
    case FLR_BF16: s = run<__nv_bfloat16>(P, Xt, y, n, p, ldn, (int)G, smem, sm_count, st, cnorm_dev, vec[5], vec[4]); break;
    case FLR_F16: s = run<__half>(P, Xt, y, n, p, ldn, (int)G, smem, sm_count, st, cnorm_dev, vec[5], vec[4]); break;
    default: return FLR_EINVAL;
  }
  if (s != FLR_OK) return s;
  unsigned char hctl[256];
  cudaError_t e = cudaMemcpyAsync(hctl, S + o_ctl, 256, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(beta_out, P.x, sizeof(double) * p, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { (void)cudaGetLastError(); return FLR_ECUDA; }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int herr;
  std::memcpy(&herr, hctl + 64, sizeof(int));
  DevStats hs;
  std::memcpy(&hs, hctl + 128, sizeof(DevStats));
  flr_status result = herr != DERR_NONE ? FLR_ETIMEOUT
                      : hs.status == -1 ? FLR_ECUDA
                                        : (flr_status)hs.status;
  if (stats) {
    stats->mm_iters = hs.mm_iters;
    stats->cg_iters = hs.cg_iters;
    stats->status = result;
    stats->grid = (int)G;
    stats->f = hs.f;
    stats->f_eps = hs.f_eps;
    stats->rel_change = hs.rel_change;
    stats->cg_relres = hs.cg_relres;
    stats->ms = ms;
    stats->refine_steps = hs.refine_steps;
    stats->reserved = 0;
    stats->est_err = estimated_error(hs);
  }
  return result;
}
