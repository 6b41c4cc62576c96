// C ABI of the fused lasso regression solver (see include/flr.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/flr.h"
#include "flr_internal.h"
#include "flr_solve.cuh"
#include "flr_batch.cuh"

using namespace flr;

namespace {

// ---------------------------------------------------------------------------
// setup kernels
// ---------------------------------------------------------------------------
// Xt[j * ldn + i] = X[i * ldx + j]  (32 x 32 tiles through shared memory)
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ X, long long n, long long p, long long ldx,
                                 T* __restrict__ Xt, long long ldn) {
  __shared__ T tile[32][33];
  const long long i0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long i = i0 + r, j = c0 + threadIdx.x;
    if (i < n && j < p) tile[r][threadIdx.x] = X[i * ldx + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long j = c0 + r, i = i0 + threadIdx.x;
    if (j < p && i < n) Xt[j * ldn + i] = tile[threadIdx.x][r];
  }
}

__global__ void fill_kernel(double* a, long long n, double v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] = v;
}

template <typename TX> __device__ __forceinline__ double widen(TX v);
template <> __device__ __forceinline__ double widen<double>(double v) { return v; }
template <> __device__ __forceinline__ double widen<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double widen<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <> __device__ __forceinline__ double widen<__half>(__half v) {
  return (double)__half2float(v);
}

// d_j = X_j^T X_j and c_j = X_j^T y in FP64 (one warp per column)
template <typename TX>
__global__ void colstats_kernel(const TX* __restrict__ Xt, const double* __restrict__ y,
                                long long n, long long p, long long ldn, double* d, double* c) {
  const int lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (j >= p) return;
  const TX* col = Xt + j * ldn;
  double sd = 0.0, sc = 0.0;
  for (long long i = lane; i < n; i += 32) {
    const double v = widen<TX>(col[i]);
    sd = fma(v, v, sd);
    sc = fma(v, y[i], sc);
  }
  sd = warp_sum(sd);
  sc = warp_sum(sc);
  if (lane == 0) { d[j] = sd; c[j] = sc; }
}

size_t dtype_size(int dt) {
  switch (dt) {
    case FLR_F64: return 8;
    case FLR_F32: return 4;
    case FLR_BF16: case FLR_F16: return 2;
    default: return 0;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct flr_handle {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  int dtype = 0;
  long long n = 0, p = 0, ldn = 0, m = 0;
  int gkind = FLR_E_CHAIN;
  long long q1 = 1, q2 = 0;
  void* Xt = nullptr;
  double *y = nullptr, *c = nullptr, *d = nullptr;
  double cnorm = 0.0;
  long long* rowptr = nullptr;
  int* col = nullptr;
  // solve workspace
  double *x = nullptr, *z = nullptr, *pb0 = nullptr, *pb1 = nullptr, *wc = nullptr, *K1 = nullptr,
         *K2 = nullptr, *binv = nullptr, *part = nullptr;
  // two-level preconditioner
  int *uf = nullptr, *cmap = nullptr, *cid = nullptr;
  double *qcinv = nullptr, *qc = nullptr, *qci = nullptr, *sc0 = nullptr, *sc1 = nullptr;
  void* ub0 = nullptr;
  void* ub1 = nullptr;
  unsigned char* ctl = nullptr;     // barrier counter, error flag, DevStats; split-barrier counters at 256
  unsigned char hctl[256];          // host copy of ctl (read once per solve)
  unsigned long long span_t0 = 0, span_t1 = 0;   // global timer span of the last solve kernel
  void* aux = nullptr;                            // workspace of another translation unit
  void (*aux_release)(void*) = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<void*> allocs;
  // batched tensor-core path (allocated on first use)
  bool batch_ready = false;
  long long ldp = 0;
  int bS = 1;
  long long bkchunk = 0;
  // split-K candidates of the batched phase A (columns per chunk), timed on the
  // first flr_solve_batch of the handle; batch_tuned once the choice is made
  long long bcand[3] = {0, 0, 0};
  int bncand = 0;
  bool batch_tuned = false;
  __nv_bfloat16* Xr = nullptr;
  double* bvec[15] = {nullptr};
  __nv_bfloat16 *Ps = nullptr, *Us = nullptr;
  float* Upart = nullptr;
  double *U0part = nullptr, *U0 = nullptr, *bred = nullptr, *blam = nullptr;
  unsigned char* bctl = nullptr;
  BatchStats* bstats = nullptr;
};

namespace {

constexpr int kMaxGrid = 512;       // grid reductions use one thread per block

// Makes `dev` current for the lifetime of the guard and restores the caller's
// device on every return path.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
    (void)cudaGetLastError();
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

flr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FLR_OK;
  if (e == cudaErrorMemoryAllocation) return FLR_ENOMEM;
  return FLR_ECUDA;
}

#define FLR_TRY(expr)                                   \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) {                            \
      (void)cudaGetLastError();                         \
      return cuda_status(_e);                           \
    }                                                   \
  } while (0)

template <typename T>
flr_status dalloc(flr_handle* h, T** out, size_t count) {
  void* ptr = nullptr;
  if (count == 0) count = 1;
  // stream-ordered: concurrent handles on other streams are not synchronised
  cudaError_t e = cudaMallocAsync(&ptr, count * sizeof(T), h->stream);
  if (e != cudaSuccess) { (void)cudaGetLastError(); return FLR_ENOMEM; }
  h->allocs.push_back(ptr);
  *out = static_cast<T*>(ptr);
  return FLR_OK;
}

void release(flr_handle* h) {
  if (!h) return;
  {
    DeviceGuard dg(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->aux && h->aux_release) h->aux_release(h->aux);
    h->aux = nullptr;
    for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
    h->allocs.clear();
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
  }
  delete h;
}

template <typename TX>
void launch_setup(flr_handle* h, const void* Xsrc, long long ldx) {
  dim3 tb(32, 8);
  dim3 grid((unsigned)((h->p + 31) / 32), (unsigned)((h->n + 31) / 32));
  using Raw = typename std::conditional<sizeof(TX) == 8, unsigned long long,
              typename std::conditional<sizeof(TX) == 4, unsigned, unsigned short>::type>::type;
  transpose_kernel<Raw><<<grid, tb, 0, h->stream>>>(static_cast<const Raw*>(Xsrc), h->n, h->p, ldx,
                                                    static_cast<Raw*>(h->Xt), h->ldn);
  const int wpb = 8;
  colstats_kernel<TX><<<(unsigned)((h->p + wpb - 1) / wpb), wpb * 32, 0, h->stream>>>(
      static_cast<const TX*>(h->Xt), h->y, h->n, h->p, h->ldn, h->d, h->c);
}

flr_status build_csr(flr_handle* h, const int64_t* edges_host, long long m) {
  const long long p = h->p;
  std::vector<std::pair<long long, long long>> pr;
  pr.reserve((size_t)m);
  for (long long e = 0; e < m; ++e) {
    long long j = edges_host[2 * e], k = edges_host[2 * e + 1];
    if (j < 0 || k < 0 || j >= p || k >= p || j == k) return FLR_EINVAL;
    if (j > k) std::swap(j, k);
    pr.emplace_back(j, k);
  }
  std::sort(pr.begin(), pr.end());
  for (size_t i = 1; i < pr.size(); ++i)
    if (pr[i] == pr[i - 1]) return FLR_EINVAL;
  std::vector<long long> rowptr((size_t)p + 1, 0);
  for (auto& e : pr) { rowptr[e.first + 1]++; rowptr[e.second + 1]++; }
  for (long long j = 0; j < p; ++j) rowptr[j + 1] += rowptr[j];
  std::vector<int> col((size_t)std::max<long long>(1, 2 * m));
  std::vector<long long> fill(rowptr.begin(), rowptr.end() - 1);
  for (auto& e : pr) {
    col[fill[e.first]++] = (int)e.second;
    col[fill[e.second]++] = (int)e.first;
  }
  for (long long j = 0; j < p; ++j) std::sort(col.begin() + rowptr[j], col.begin() + rowptr[j + 1]);
  flr_status s;
  if ((s = dalloc(h, &h->rowptr, (size_t)p + 1)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->col, (size_t)std::max<long long>(1, 2 * m))) != FLR_OK) return s;
  if ((s = dalloc(h, &h->wc, (size_t)std::max<long long>(1, 2 * m))) != FLR_OK) return s;
  FLR_TRY(cudaMemcpyAsync(h->rowptr, rowptr.data(), sizeof(long long) * (p + 1), cudaMemcpyHostToDevice,
                          h->stream));
  FLR_TRY(cudaMemcpyAsync(h->col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, h->stream));
  FLR_TRY(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
  return FLR_OK;
}

// Largest dynamic shared memory a launch of `kern` may request on `dev`: the
// per-block opt-in limit minus the kernel's static shared memory.
cudaError_t max_dynamic_smem(const void* kern, int dev, int* out) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  *out = optin - (int)fa.sharedSizeBytes;
  return cudaSuccess;
}

template <typename TX, int GK, bool CH = false>
flr_status launch_solve_t(flr_handle* h, SolveParams& P, int G, size_t smem) {
  auto kern = mm_solve_kernel<TX, GK, CH>;
  // The attribute is per kernel, shared by every thread of the process: set it
  // to the most the device allows next to the kernel's static shared memory
  // (the same value from every caller), never to this launch's size, which a
  // concurrent solve could lower before this launch.
  int dyn_max = 0;
  FLR_TRY(max_dynamic_smem((const void*)kern, h->device, &dyn_max));
  if (smem > (size_t)dyn_max) return FLR_ENOTIMPL;
  FLR_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
  // slab columns after the TMEM ones resident in shared memory (x_smem = 0), the rest streamed
  if (P.ws != 0) {
    P.ws = resident_columns(P.w - P.wt, P.ldn, sizeof(TX), smem, dyn_max);
    if (P.ws > 0) smem = (smem + 15) / 16 * 16 + (size_t)P.ws * (size_t)P.ldn * sizeof(TX);
  }
  int nb = 0;
  FLR_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem));
  if (nb < 1 || G > nb * h->sm_count) return FLR_ENOTIMPL;
  void* args[] = {(void*)&P};
  FLR_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(kThreads), args, smem,
                                      h->stream));
  return FLR_OK;
}

flr_status launch_solve(flr_handle* h, SolveParams& P, int G, size_t smem) {
  const int gk = h->gkind == FLR_E_EDGES ? GK_CSR : GK_STENCIL;
  if (P.chunked) {   // one-pass chunked Q-apply (32- and 16-bit X)
    flr_status s = FLR_EINVAL;
    switch (h->dtype) {
      case FLR_F32: s = gk ? launch_solve_t<float, GK_CSR, true>(h, P, G, smem)
                           : launch_solve_t<float, GK_STENCIL, true>(h, P, G, smem); break;
      case FLR_BF16: s = gk ? launch_solve_t<__nv_bfloat16, GK_CSR, true>(h, P, G, smem)
                            : launch_solve_t<__nv_bfloat16, GK_STENCIL, true>(h, P, G, smem); break;
      case FLR_F16: s = gk ? launch_solve_t<__half, GK_CSR, true>(h, P, G, smem)
                           : launch_solve_t<__half, GK_STENCIL, true>(h, P, G, smem); break;
      default: break;
    }
    return s;
  }
  switch (h->dtype) {
    case FLR_F64: return gk ? launch_solve_t<double, GK_CSR>(h, P, G, smem)
                            : launch_solve_t<double, GK_STENCIL>(h, P, G, smem);
    case FLR_F32: return gk ? launch_solve_t<float, GK_CSR>(h, P, G, smem)
                            : launch_solve_t<float, GK_STENCIL>(h, P, G, smem);
    case FLR_BF16: return gk ? launch_solve_t<__nv_bfloat16, GK_CSR>(h, P, G, smem)
                             : launch_solve_t<__nv_bfloat16, GK_STENCIL>(h, P, G, smem);
    case FLR_F16: return gk ? launch_solve_t<__half, GK_CSR>(h, P, G, smem)
                            : launch_solve_t<__half, GK_STENCIL>(h, P, G, smem);
    case FLR_IDENTITY: return gk ? launch_solve_t<IdX, GK_CSR>(h, P, G, smem)
                                 : launch_solve_t<IdX, GK_STENCIL>(h, P, G, smem);
  }
  return FLR_EINVAL;
}


flr_status batch_prepare(flr_handle* h) {
  if (h->batch_ready) return FLR_OK;
  flr_status s;
  const long long n = h->n, p = h->p;
  h->ldp = (p + 7) / 8 * 8;
  const long long mtiles = (n + kTM - 1) / kTM;
  // phase A splits the reduction over p into S chunks so that about one work item
  // (row tile, chunk) falls to each SM; the autotuner also tries half and twice
  // that chunk length
  int S = (int)std::max<long long>(1, (long long)h->sm_count / mtiles);
  long long kchunk = (h->ldp + S - 1) / S;
  kchunk = (kchunk + 63) / 64 * 64;
  S = (int)((h->ldp + kchunk - 1) / kchunk);
  h->bS = S;
  h->bkchunk = kchunk;
  int Smax = S;
  h->bncand = 0;
  for (long long kc : {kchunk, (kchunk / 2 + 63) / 64 * 64, kchunk * 2}) {
    bool dup = kc < 64 || (kc > h->ldp && kc != kchunk);
    for (int i = 0; i < h->bncand; ++i) dup = dup || ((h->ldp + kc - 1) / kc == (h->ldp + h->bcand[i] - 1) / h->bcand[i]);
    if (dup) continue;
    h->bcand[h->bncand++] = kc;
    Smax = std::max<int>(Smax, (int)((h->ldp + kc - 1) / kc));
  }
  if ((s = dalloc(h, &h->Xr, (size_t)(n * h->ldp))) != FLR_OK) return s;
  for (int i = 0; i < 15; ++i)
    if ((s = dalloc(h, &h->bvec[i], (size_t)kNRMax * p)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->Ps, (size_t)kSlices * kNRMax * h->ldp)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->Us, (size_t)kSlices * kNRMax * h->ldn)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->Upart, (size_t)Smax * kNRMax * n)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->U0part, (size_t)Smax * kNRMax * n)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->U0, (size_t)kNRMax * n)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->bred, (size_t)kRedSlots * 4 * kNRMax)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->blam, (size_t)2 * kNRMax)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->bctl, 256)) != FLR_OK) return s;
  if ((s = dalloc(h, &h->bstats, (size_t)kNRMax)) != FLR_OK) return s;
  // row-major copy of X (the A operand of X P) from the column-major copy
  FLR_TRY(cudaMemsetAsync(h->Xr, 0, sizeof(__nv_bfloat16) * n * h->ldp, h->stream));
  FLR_TRY(cudaMemsetAsync(h->Ps, 0, sizeof(__nv_bfloat16) * kSlices * kNRMax * h->ldp, h->stream));
  FLR_TRY(cudaMemsetAsync(h->Us, 0, sizeof(__nv_bfloat16) * kSlices * kNRMax * h->ldn, h->stream));
  dim3 tb(32, 8);
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((p + 31) / 32));
  transpose_kernel<unsigned short><<<grid, tb, 0, h->stream>>>(
      static_cast<const unsigned short*>(h->Xt), p, n, h->ldn,
      reinterpret_cast<unsigned short*>(h->Xr), h->ldp);
  FLR_TRY(cudaGetLastError());
  h->batch_ready = true;
  return FLR_OK;
}

flr_status batch_group(flr_handle* h, int K, const double* l1, const double* l2, double eps,
                       double tol, const flr_opts& o, double* betas, int io_mem,
                       double* objectives, flr_stats* stats);

// The autotuner: on the first batched solve of a handle, time one launch per
// split-K candidate (one MM iteration, its FP64 passes and kTuneCG lockstep CG
// iterations of the caller's first RHS group and options) and keep the fastest.
constexpr int kTuneCG = 24;
flr_status batch_tune(flr_handle* h, int K, const double* l1, const double* l2, double eps, double tol,
                      const flr_opts& o) {
  flr_status s = batch_prepare(h);
  if (s != FLR_OK || h->batch_tuned) return s;
  h->batch_tuned = true;
  if (h->bncand <= 1) return FLR_OK;
  flr_opts t = o;
  t.max_mm = 1;
  t.max_cg = kTuneCG;
  t.min_cg = kTuneCG;
  t.tol_cg = 1e-300;
  t.tol_cg_rel = 0.0;
  t.max_refine = 0;
  std::vector<double> b((size_t)K * h->p);
  std::vector<flr_stats> st((size_t)K);
  float best = 0.f;
  long long kbest = h->bkchunk;
  for (int c = 0; c < h->bncand; ++c) {
    h->bkchunk = h->bcand[c];
    h->bS = (int)((h->ldp + h->bkchunk - 1) / h->bkchunk);
    s = batch_group(h, K, l1, l2, eps, tol, t, b.data(), FLR_MEM_HOST, nullptr, st.data());
    if (s == FLR_EINVAL || s == FLR_ECUDA || s == FLR_ENOMEM || s == FLR_ENOTIMPL || s == FLR_ETIMEOUT)
      return s;
    if (c == 0 || st[0].ms < best) { best = (float)st[0].ms; kbest = h->bkchunk; }
  }
  h->bkchunk = kbest;
  h->bS = (int)((h->ldp + kbest - 1) / kbest);
  return FLR_OK;
}

// Solve K <= 64 problems in one launch of mm_batch_kernel.
flr_status batch_group(flr_handle* h, int K, const double* l1, const double* l2, double eps,
                       double tol, const flr_opts& o, double* betas, int io_mem,
                       double* objectives, flr_stats* stats) {
  flr_status s = batch_prepare(h);
  if (s != FLR_OK) return s;
  const int NR = K <= 32 ? 32 : 64;
  const long long n = h->n, p = h->p;
  std::vector<double> lam((size_t)2 * kNRMax, 0.0);
  for (int k = 0; k < K; ++k) { lam[k] = l1[k]; lam[kNRMax + k] = l2[k]; }
  FLR_TRY(cudaMemcpyAsync(h->blam, lam.data(), sizeof(double) * 2 * kNRMax, cudaMemcpyHostToDevice,
                          h->stream));
  FLR_TRY(cudaMemsetAsync(h->bred, 0, sizeof(double) * kRedSlots * 4 * kNRMax, h->stream));
  FLR_TRY(cudaMemsetAsync(h->bctl, 0, 256, h->stream));
  FLR_TRY(cudaMemsetAsync(h->bstats, 0xff, sizeof(BatchStats) * kNRMax, h->stream));
  BatchParams P{};
  P.Xr = h->Xr; P.Xt = static_cast<const __nv_bfloat16*>(h->Xt);
  P.n = n; P.p = p; P.ldp = h->ldp; P.ldn = h->ldn;
  P.q2 = h->gkind == FLR_E_LATTICE ? h->q2 : p;
  P.K = K; P.NR = NR;
  P.y = h->y; P.c = h->c; P.d = h->d; P.cnorm = h->cnorm > 0 ? h->cnorm : 1.0;
  P.lam1 = h->blam; P.lam2 = h->blam + kNRMax;
  P.eps = eps; P.tol = tol; P.tol_cg = o.tol_cg > 0.0 ? o.tol_cg : tol;
  P.tol_cg_rel = o.tol_cg_rel;
  P.max_mm = o.max_mm; P.max_cg = o.max_cg; P.min_cg = o.min_cg;
  P.S = h->bS; P.kchunk = h->bkchunk;
  double** v = h->bvec;
  P.x = v[0]; P.r = v[1]; P.z = v[2]; P.pb0 = v[3]; P.pb1 = v[4]; P.q = v[5]; P.la = v[6];
  P.wl = v[7]; P.wr = v[8]; P.wu = v[9]; P.wd = v[10]; P.idg = v[11]; P.t0 = v[12];
  P.lmul = v[13]; P.dinv = v[14];
  {
    int pc = o.precond;
    if (pc == FLR_PC_AUTO) pc = FLR_PC_TRIDIAG;
    P.precond = pc == FLR_PC_TRIDIAG ? PC_TRIDIAG : pc == FLR_PC_PAPER ? PC_PAPER : PC_JACOBI;
  }
  P.max_refine = o.max_refine;
  P.Ps = h->Ps; P.Us = h->Us; P.Upart = h->Upart; P.U0part = h->U0part; P.U0 = h->U0;
  P.red = h->bred;
  P.bar = reinterpret_cast<unsigned*>(h->bctl);
  P.err = reinterpret_cast<int*>(h->bctl + 64);
  P.stats = h->bstats;
  P.timeout = o.wait_cycles > 0 ? o.wait_cycles : (1LL << 33);
  const size_t smem = batch_smem_bytes(NR);
  int dyn_max = 0;
  FLR_TRY(max_dynamic_smem((const void*)mm_batch_kernel, h->device, &dyn_max));
  if (smem > (size_t)dyn_max) return FLR_ENOTIMPL;
  FLR_TRY(cudaFuncSetAttribute(mm_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
  int nb = 0;
  FLR_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mm_batch_kernel, kBT, smem));
  if (nb < 1) return FLR_ENOTIMPL;
  const long long ntiles = (p + kTM - 1) / kTM;
  const long long mtiles = (n + kTM - 1) / kTM;
  long long G = std::max<long long>(ntiles, mtiles * h->bS);
  G = std::max<long long>(1, std::min<long long>({G, (long long)h->sm_count * nb, (long long)h->sm_count}));
  void* args[] = {(void*)&P};
  FLR_TRY(cudaEventRecord(h->ev0, h->stream));
  FLR_TRY(cudaLaunchCooperativeKernel((const void*)mm_batch_kernel, dim3((unsigned)G), dim3(kBT), args,
                                      smem, h->stream));
  FLR_TRY(cudaEventRecord(h->ev1, h->stream));
  std::vector<BatchStats> hs((size_t)K);
  unsigned char hctl[256];
  FLR_TRY(cudaMemcpyAsync(hs.data(), h->bstats, sizeof(BatchStats) * K, cudaMemcpyDeviceToHost, h->stream));
  FLR_TRY(cudaMemcpyAsync(hctl, h->bctl, 256, cudaMemcpyDeviceToHost, h->stream));
  std::vector<double> hb((size_t)K * p);
  FLR_TRY(cudaMemcpyAsync(hb.data(), P.x, sizeof(double) * K * p, cudaMemcpyDeviceToHost, h->stream));
  FLR_TRY(cudaStreamSynchronize(h->stream));
  if (io_mem == FLR_MEM_HOST) {
    std::memcpy(betas, hb.data(), sizeof(double) * K * p);
  } else {
    FLR_TRY(cudaMemcpyAsync(betas, hb.data(), sizeof(double) * K * p, cudaMemcpyHostToDevice, h->stream));
    FLR_TRY(cudaStreamSynchronize(h->stream));
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  int herr;
  std::memcpy(&herr, hctl + 64, sizeof(int));
  flr_status first = FLR_OK;
  const long long q2 = P.q2;
  for (int k = 0; k < K; ++k) {
    flr_status sk = herr != DERR_NONE ? FLR_ETIMEOUT
                    : hs[k].status == -1 ? FLR_ECUDA : (flr_status)hs[k].status;
    // f_eps = f - lam1 sum eps log(1+|b|/eps) - lam2 sum_E eps log(1+|d|/eps)  (Eq. pert)
    const double* bk = hb.data() + (size_t)k * p;
    double g1 = 0.0, g2 = 0.0;
    for (long long j = 0; j < p; ++j) {
      g1 += eps * std::log1p(std::fabs(bk[j]) / eps);
      if ((j % q2) != q2 - 1 && j + 1 < p) g2 += eps * std::log1p(std::fabs(bk[j] - bk[j + 1]) / eps);
      if (j + q2 < p) g2 += eps * std::log1p(std::fabs(bk[j] - bk[j + q2]) / eps);
    }
    if (objectives) objectives[k] = hs[k].f;
    if (stats) {
      stats[k].mm_iters = hs[k].mm_iters;
      stats[k].cg_iters = hs[k].cg_iters;
      stats[k].status = sk;
      stats[k].grid = (int)G;
      stats[k].f = hs[k].f;
      stats[k].f_eps = hs[k].f - l1[k] * g1 - l2[k] * g2;
      stats[k].rel_change = hs[k].rel_change;
      stats[k].cg_relres = hs[k].cg_relres;
      stats[k].ms = ms;
      stats[k].refine_steps = hs[k].refine_steps;
      stats[k].reserved = 0;
      DevStats ds{};
      ds.f = hs[k].f;
      ds.f_eps = stats[k].f_eps;
      ds.rel_change = hs[k].rel_change;
      ds.rel_prev = hs[k].rel_prev;
      stats[k].est_err = estimated_error(ds);
    }
    if (sk != FLR_OK && first == FLR_OK) first = sk;
  }
  return first;
}

}  // namespace

// ---------------------------------------------------------------------------
// public API
// ---------------------------------------------------------------------------
extern "C" {

void flr_default_opts(flr_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_mm = 10000;
  o->max_cg = 10000;
  o->min_cg = 1;
  o->precond = FLR_PC_AUTO;
  o->tol_cg = 0.0;
  o->grid = 0;
}

const char* flr_strerror(int32_t s) {
  switch (s) {
    case FLR_OK: return "FLR_OK: success";
    case FLR_EINVAL: return "FLR_EINVAL: invalid argument";
    case FLR_ENOMEM: return "FLR_ENOMEM: out of memory";
    case FLR_ECUDA: return "FLR_ECUDA: CUDA runtime error";
    case FLR_ENOTCONV: return "FLR_ENOTCONV: MM iteration cap reached before the stop test held";
    case FLR_EBREAKDOWN: return "FLR_EBREAKDOWN: CG breakdown (p^T Q p <= 0)";
    case FLR_ENONFINITE: return "FLR_ENONFINITE: non-finite value";
    case FLR_ETIMEOUT: return "FLR_ETIMEOUT: a bounded device-side wait gave up";
    case FLR_ENOTIMPL: return "FLR_ENOTIMPL: combination not implemented";
    case FLR_ESCRATCH: return "FLR_ESCRATCH: problem too large for the static scratch of flr_solve_noalloc";
    default: return "unknown flr_status";
  }
}

flr_status flr_create(const void* X, int32_t dtype, int64_t n, int64_t p, int64_t ldx,
                      const double* y, const flr_graph* E, int32_t mem, void* stream,
                      flr_t* out) {
  if (!out) return FLR_EINVAL;
  *out = nullptr;
  const bool ident = dtype == FLR_IDENTITY;
  if (!y || !E || n < 1 || p < 1) return FLR_EINVAL;
  if (ident ? (X != nullptr || n != p) : (!X || ldx < p || dtype_size(dtype) == 0)) return FLR_EINVAL;
  if (mem != FLR_MEM_DEVICE && mem != FLR_MEM_HOST) return FLR_EINVAL;
  if (p >= (int64_t)INT32_MAX || n >= (int64_t)INT32_MAX) return FLR_ENOTIMPL;
  long long q1 = 1, q2 = p, m = 0;
  switch (E->kind) {
    case FLR_E_CHAIN: m = p - 1; break;
    case FLR_E_LATTICE:
      if (E->q1 < 1 || E->q2 < 1 || E->q1 * E->q2 != p) return FLR_EINVAL;
      q1 = E->q1; q2 = E->q2;
      m = q1 * (q2 - 1) + (q1 - 1) * q2;
      break;
    case FLR_E_EDGES:
      if (E->m < 0 || (E->m > 0 && !E->edges)) return FLR_EINVAL;
      m = E->m;
      break;
    default: return FLR_EINVAL;
  }
  flr_handle* h = new (std::nothrow) flr_handle();
  if (!h) return FLR_ENOMEM;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  h->stream = static_cast<cudaStream_t>(stream);
  h->dtype = dtype;
  h->n = n; h->p = p; h->m = m;
  h->gkind = E->kind; h->q1 = q1; h->q2 = q2;
  const size_t es = ident ? 8 : dtype_size(dtype);
  const long long vec = 16 / (long long)es;
  h->ldn = ident ? vec : (n + vec - 1) / vec * vec;   // X = I keeps no n-vector accumulators
  flr_status s = FLR_OK;
  auto fail = [&](flr_status st) { release(h); return st; };

  // graph (validated on the host)
  if (E->kind == FLR_E_EDGES) {
    std::vector<int64_t> eh((size_t)(2 * m));
    if (m > 0) {
      if (mem == FLR_MEM_HOST) std::memcpy(eh.data(), E->edges, sizeof(int64_t) * 2 * m);
      else if (cudaMemcpyAsync(eh.data(), E->edges, sizeof(int64_t) * 2 * m, cudaMemcpyDeviceToHost,
                               h->stream) != cudaSuccess ||
               cudaStreamSynchronize(h->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(FLR_EINVAL);
      }
    }
    if ((s = build_csr(h, eh.data(), m)) != FLR_OK) return fail(s);
  }
  // buffers
  const size_t P = (size_t)p;
  if (!ident &&
      (s = dalloc(h, reinterpret_cast<unsigned char**>(&h->Xt), (size_t)(p * h->ldn) * es)) != FLR_OK)
    return fail(s);
  if ((s = dalloc(h, &h->y, (size_t)n)) != FLR_OK) return fail(s);
  if ((s = dalloc(h, &h->c, P)) != FLR_OK) return fail(s);
  if ((s = dalloc(h, &h->d, P)) != FLR_OK) return fail(s);
  double** vecs[] = {&h->x, &h->z, &h->pb0, &h->pb1, &h->binv,
                     &h->qcinv, &h->qc, &h->qci, &h->sc0, &h->sc1};
  for (double** v : vecs)
    if ((s = dalloc(h, v, P)) != FLR_OK) return fail(s);
  int** ivecs[] = {&h->uf, &h->cmap, &h->cid};
  for (int** v : ivecs)
    if ((s = dalloc(h, v, P)) != FLR_OK) return fail(s);
  if ((s = dalloc(h, &h->K1, P * kMaxLevels)) != FLR_OK) return fail(s);
  if ((s = dalloc(h, &h->K2, P * kMaxLevels)) != FLR_OK) return fail(s);
  if (!h->wc && (s = dalloc(h, &h->wc, 1)) != FLR_OK) return fail(s);
  // u buffers hold doubles (the FP64 refinement pass) and floats (FP32 CG products)
  if ((s = dalloc(h, reinterpret_cast<unsigned char**>(&h->ub0), (size_t)h->ldn * 8 * kUR)) != FLR_OK) return fail(s);
  if ((s = dalloc(h, reinterpret_cast<unsigned char**>(&h->ub1), (size_t)h->ldn * 8 * kUR)) != FLR_OK) return fail(s);
  if ((s = dalloc(h, &h->part, (size_t)2 * kNF * kMaxGrid)) != FLR_OK) return fail(s);
  if ((s = dalloc(h, &h->ctl, 512)) != FLR_OK) return fail(s);
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) return fail(FLR_ECUDA);

  if (ident) {   // X = I: X^T y = y, diag(X^T X) = 1
    const cudaMemcpyKind kd = mem == FLR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(h->y, y, sizeof(double) * n, kd, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->c, y, sizeof(double) * n, kd, h->stream) != cudaSuccess)
      return fail(FLR_ECUDA);
    fill_kernel<<<(unsigned)std::min<long long>((p + 255) / 256, 1024), 256, 0, h->stream>>>(h->d, p, 1.0);
    std::vector<double> yh((size_t)n);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(yh.data(), h->c, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return fail(FLR_ECUDA);
    double s2 = 0.0;
    for (double v : yh) s2 += v * v;
    h->cnorm = std::sqrt(s2);
    if (!std::isfinite(h->cnorm)) return fail(FLR_ENONFINITE);
    *out = h;
    return FLR_OK;
  }
  // X -> column-major copy (padding rows are zero), y, then X^T y and diag(X^T X)
  if (cudaMemsetAsync(h->Xt, 0, (size_t)(p * h->ldn) * es, h->stream) != cudaSuccess) return fail(FLR_ECUDA);
  const void* Xdev = X;
  void* staging = nullptr;
  if (mem == FLR_MEM_HOST) {
    if (cudaMallocAsync(&staging, (size_t)(n * ldx) * es, h->stream) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(FLR_ENOMEM);
    }
    if (cudaMemcpyAsync(staging, X, (size_t)(n * ldx) * es, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
      cudaFreeAsync(staging, h->stream);
      return fail(FLR_ECUDA);
    }
    Xdev = staging;
  }
  if (cudaMemcpyAsync(h->y, y, sizeof(double) * n,
                      mem == FLR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                      h->stream) != cudaSuccess) {
    if (staging) cudaFreeAsync(staging, h->stream);
    return fail(FLR_ECUDA);
  }
  switch (dtype) {
    case FLR_F64: launch_setup<double>(h, Xdev, ldx); break;
    case FLR_F32: launch_setup<float>(h, Xdev, ldx); break;
    case FLR_BF16: launch_setup<__nv_bfloat16>(h, Xdev, ldx); break;
    case FLR_F16: launch_setup<__half>(h, Xdev, ldx); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (staging) cudaFreeAsync(staging, h->stream);
  if (e != cudaSuccess) return fail(cuda_status(e));
  std::vector<double> ch((size_t)p);
  if (cudaMemcpyAsync(ch.data(), h->c, sizeof(double) * p, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return fail(FLR_ECUDA);
  double s2 = 0.0;
  for (double v : ch) s2 += v * v;
  h->cnorm = std::sqrt(s2);
  if (!std::isfinite(h->cnorm)) return fail(FLR_ENONFINITE);
  *out = h;
  return FLR_OK;
}

flr_status flr_solve(flr_t h, double lambda1, double lambda2, double eps, double tol,
                     const flr_opts* opts, const double* beta_init, double* beta_out,
                     int32_t io_mem, flr_stats* stats) {
  if (!h || !beta_out) return FLR_EINVAL;
  if (!(lambda1 >= 0.0) || !(lambda2 >= 0.0) || !(eps > 0.0) || !(tol > 0.0)) return FLR_EINVAL;
  if (!std::isfinite(lambda1) || !std::isfinite(lambda2) || !std::isfinite(eps)) return FLR_EINVAL;
  if (io_mem != FLR_MEM_DEVICE && io_mem != FLR_MEM_HOST) return FLR_EINVAL;
  flr_opts o;
  flr_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_mm < 0 || o.max_cg < 0 || o.min_cg < 0 || o.tol_cg < 0.0 || o.wait_cycles < 0 ||
      o.max_refine < 0 || o.x_smem < -1 || o.x_smem > 1 ||
      !(o.tol_cg_rel >= 0.0))
    return FLR_EINVAL;
  DeviceGuard dg(h->device);

  int precond = o.precond;
  if (precond == FLR_PC_AUTO) precond = FLR_PC_TWOLEVEL;
  if (precond != FLR_PC_JACOBI && precond != FLR_PC_TRIDIAG && precond != FLR_PC_PAPER &&
      precond != FLR_PC_TWOLEVEL)
    return FLR_EINVAL;
  if ((precond == FLR_PC_TRIDIAG || precond == FLR_PC_PAPER) && h->gkind == FLR_E_EDGES) return FLR_ENOTIMPL;

  // grid: one block per SM at most; fewer for small problems
  const bool ident = h->dtype == FLR_IDENTITY;
  const long long work = ident ? h->p : h->n * h->p;
  const long long per_block = ident ? 256 : h->dtype == FLR_F64 ? 8192 : 65536;
  long long G = o.grid > 0 ? o.grid : (work + per_block - 1) / per_block;
  G = std::max<long long>(1, std::min<long long>({G, (long long)h->sm_count, (long long)kMaxGrid, h->p}));
  long long w = (h->p + G - 1) / G;
  G = (h->p + w - 1) / w;
  if (w > 8192) return FLR_ENOTIMPL;
  int levels = 0;
  while ((1LL << levels) < w) ++levels;
  const long long wpad = (w + 3) / 4 * 4;
  const int V = ident ? XT<IdX>::V : (int)(16 / dtype_size(h->dtype));
  const long long q2p = h->gkind == FLR_E_LATTICE ? h->q2 : h->p;
  // X on chip (x_smem = 0): the leading columns of every slab in TMEM, the next
  // ones in shared memory (sized at launch), the rest streamed twice per CG
  // iteration; x_smem = 1: the chunked one-pass Q-apply (32- and 16-bit X)
  const bool chunked = !ident && h->dtype != FLR_F64 && o.x_smem == 1;
  const int tct = (o.x_smem == 0 && !ident && !chunked) ? tmem_cells(h->n, (int)dtype_size(h->dtype)) : 0;
  const long long trows = tct > 0 ? (h->n + 127) / 128 * 128 : 0;
  const size_t smem = solve_smem_bytes(h->ldn, wpad, V, halo_entries(wpad, q2p, h->p), trows);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (smem > (size_t)smem_max) return FLR_ENOTIMPL;

  unsigned* bar = reinterpret_cast<unsigned*>(h->ctl);
  int* err = reinterpret_cast<int*>(h->ctl + 64);
  DevStats* dst = reinterpret_cast<DevStats*>(h->ctl + 128);
  FLR_TRY(cudaMemsetAsync(h->ctl, 0, 128, h->stream));
  FLR_TRY(cudaMemsetAsync(h->ctl + 128, 0xff, 128, h->stream));   // status -1 until written
  FLR_TRY(cudaMemsetAsync(h->ctl + 256, 0, 256, h->stream));       // split-barrier counters
  const size_t accsz = (size_t)h->ldn * 8 * kUR;
  FLR_TRY(cudaMemsetAsync(h->ub0, 0, accsz, h->stream));
  FLR_TRY(cudaMemsetAsync(h->ub1, 0, accsz, h->stream));
  const double* binit = nullptr;
  if (beta_init) {
    FLR_TRY(cudaMemcpyAsync(h->x, beta_init, sizeof(double) * h->p,
                            io_mem == FLR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            h->stream));
    binit = h->x;
  }

  SolveParams P{};
  P.Xt = h->Xt; P.n = h->n; P.p = h->p; P.ldn = h->ldn;
  P.y = h->y; P.c = h->c; P.d = h->d; P.cnorm = h->cnorm > 0 ? h->cnorm : 1.0;
  P.q2 = h->gkind == FLR_E_LATTICE ? h->q2 : h->p;
  P.rowptr = h->rowptr; P.col = h->col;
  P.lam1 = lambda1; P.lam2 = lambda2; P.eps = eps; P.tol = tol;
  P.tol_cg = o.tol_cg > 0.0 ? o.tol_cg : tol;
  P.tol_cg_rel = o.tol_cg_rel;
  P.max_mm = o.max_mm; P.max_cg = o.max_cg; P.min_cg = o.min_cg; P.precond = precond;
  P.max_refine = o.max_refine;
  P.ws = (o.x_smem == 0 && !ident && !chunked) ? 1 : 0;   // 1: size the resident columns at launch
  P.chunked = chunked ? 1 : 0;
  P.cbar = reinterpret_cast<unsigned*>(h->ctl + 256);
  P.tct = tct;
  P.wt = tct > 0 ? tct * (4 / (int)dtype_size(h->dtype)) : 0;
  P.w = w; P.wpad = wpad; P.levels = levels;
  P.beta_init = binit;
  P.x = h->x; P.z = h->z; P.pb0 = h->pb0; P.pb1 = h->pb1; P.wc = h->wc;
  P.K1 = h->K1; P.K2 = h->K2; P.binv = h->binv;
  P.uf = h->uf; P.cmap = h->cmap; P.cid = h->cid; P.ncomp = reinterpret_cast<int*>(h->ctl + 96);
  P.qcinv = h->qcinv; P.qc = h->qc; P.qci = h->qci; P.sc0 = h->sc0; P.sc1 = h->sc1;
  P.ub0 = h->ub0; P.ub1 = h->ub1; P.part = h->part;
  P.bar = bar; P.err = err; P.stats = dst;
  P.timeout = o.wait_cycles > 0 ? o.wait_cycles : (1LL << 33);   // ~4 s of SM clock
  P.inject_stall = o.inject_stall;

  FLR_TRY(cudaEventRecord(h->ev0, h->stream));
  flr_status ls = launch_solve(h, P, (int)G, smem);
  if (ls != FLR_OK) return ls;
  FLR_TRY(cudaEventRecord(h->ev1, h->stream));
  FLR_TRY(cudaMemcpyAsync(h->hctl, h->ctl, 256, cudaMemcpyDeviceToHost, h->stream));
  FLR_TRY(cudaMemcpyAsync(beta_out, h->x, sizeof(double) * h->p,
                          io_mem == FLR_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          h->stream));
  FLR_TRY(cudaStreamSynchronize(h->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  const int herr = *reinterpret_cast<const int*>(h->hctl + 64);
  const DevStats* hs = reinterpret_cast<const DevStats*>(h->hctl + 128);
  flr_status st = herr != DERR_NONE ? FLR_ETIMEOUT
                  : hs->status == -1 ? FLR_ECUDA            // the kernel did not finish its work
                                     : (flr_status)hs->status;
  if (stats) {
    stats->mm_iters = hs->mm_iters;
    stats->cg_iters = hs->cg_iters;
    stats->status = st;
    stats->grid = (int)G;
    stats->f = hs->f;
    stats->f_eps = hs->f_eps;
    stats->rel_change = hs->rel_change;
    stats->cg_relres = hs->cg_relres;
    stats->ms = ms;
    stats->refine_steps = hs->refine_steps;
    stats->reserved = 0;
    stats->est_err = estimated_error(*hs);
  }
  h->span_t0 = hs->t0_ns;
  h->span_t1 = hs->t1_ns;
  return st;
}

flr_status flr_solve_batch(flr_t h, int32_t K, const double* lambda1, const double* lambda2,
                           double eps, double tol, const flr_opts* opts, double* betas,
                           int32_t io_mem, double* objectives, flr_stats* stats) {
  if (!h || K < 0 || (K > 0 && (!lambda1 || !lambda2 || !betas))) return FLR_EINVAL;
  if (!(eps > 0.0) || !(tol > 0.0) || (io_mem != FLR_MEM_DEVICE && io_mem != FLR_MEM_HOST)) return FLR_EINVAL;
  for (int k = 0; k < K; ++k)
    if (!(lambda1[k] >= 0.0) || !(lambda2[k] >= 0.0) || !std::isfinite(lambda1[k]) ||
        !std::isfinite(lambda2[k]))
      return FLR_EINVAL;
  flr_opts o;
  flr_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_mm < 0 || o.max_cg < 0 || o.min_cg < 0 || o.tol_cg < 0.0 || o.wait_cycles < 0 ||
      o.max_refine < 0 || !(o.tol_cg_rel >= 0.0))
    return FLR_EINVAL;
  DeviceGuard dg(h->device);
  // tensor-core multi-RHS path: BF16 X, chain/lattice, a diagonal or per-tile tridiagonal preconditioner
  const bool tc_path = h->dtype == FLR_BF16 && h->gkind != FLR_E_EDGES && K >= 1 &&
                       (o.precond == FLR_PC_AUTO || o.precond == FLR_PC_JACOBI ||
                        o.precond == FLR_PC_TRIDIAG || o.precond == FLR_PC_PAPER);
  if (tc_path) {
    flr_status first = batch_tune(h, std::min(kNRMax, (int)K), lambda1, lambda2, eps, tol, o);
    if (first != FLR_OK) return first;
    for (int k0 = 0; k0 < K; k0 += kNRMax) {
      const int kg = std::min(kNRMax, K - k0);
      flr_status s = batch_group(h, kg, lambda1 + k0, lambda2 + k0, eps, tol, o,
                                 betas + (size_t)k0 * h->p, io_mem,
                                 objectives ? objectives + k0 : nullptr, stats ? stats + k0 : nullptr);
      if (s == FLR_EINVAL || s == FLR_ECUDA || s == FLR_ENOMEM || s == FLR_ENOTIMPL) return s;
      if (s != FLR_OK && first == FLR_OK) first = s;
    }
    return first;
  }
  flr_status first = FLR_OK;
  for (int k = 0; k < K; ++k) {
    flr_stats st{};
    flr_status s = flr_solve(h, lambda1[k], lambda2[k], eps, tol, opts, nullptr,
                             betas + (size_t)k * h->p, io_mem, &st);
    if (objectives) objectives[k] = st.f;
    if (stats) stats[k] = st;
    if (s != FLR_OK && first == FLR_OK) first = s;
    if (s == FLR_EINVAL || s == FLR_ECUDA || s == FLR_ENOMEM) return s;
  }
  return first;
}

void flr_destroy(flr_t h) { release(h); }

}  // extern "C"

int flr_min_grid(flr_t h) {
  if (!h || h->dtype == FLR_IDENTITY) return 1;
  int dyn_max = 0;
  if (max_dynamic_smem((const void*)mm_solve_kernel<float, GK_STENCIL>, h->device, &dyn_max) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1;
  }
  const int V = (int)(16 / dtype_size(h->dtype));
  const long long q2p = h->gkind == FLR_E_LATTICE ? h->q2 : h->p;
  // as flr_solve with the default x_smem: TMEM row partials when X fits in TMEM
  const int tct = h->dtype != FLR_F64 ? tmem_cells(h->n, (int)dtype_size(h->dtype)) : 0;
  const long long trows = tct > 0 ? (h->n + 127) / 128 * 128 : 0;
  for (long long G = 1; G <= h->sm_count && G <= kMaxGrid; ++G) {
    const long long w = (h->p + G - 1) / G;
    if (w > 8192) continue;
    const long long wpad = (w + 3) / 4 * 4;
    // (the margin covers the other kernel instances' slightly different static shared memory)
    if (solve_smem_bytes(h->ldn, wpad, V, halo_entries(wpad, q2p, h->p), trows) + 1024 <= (size_t)dyn_max)
      return (int)G;
  }
  return -1;
}

void flr_kernel_span(flr_t h, unsigned long long* t0, unsigned long long* t1) {
  *t0 = h ? h->span_t0 : 0;
  *t1 = h ? h->span_t1 : 0;
}

bool flr_get_view(flr_t h, flr_view* v) {
  if (!h || !v) return false;
  v->device = h->device;
  v->sm_count = h->sm_count;
  v->stream = h->stream;
  v->dtype = h->dtype;
  v->n = h->n; v->p = h->p; v->ldn = h->ldn; v->m = h->m;
  v->gkind = h->gkind;
  v->q2 = h->gkind == FLR_E_LATTICE ? h->q2 : h->p;
  v->Xt = h->Xt;
  v->y = h->y; v->c = h->c; v->d = h->d;
  v->cnorm = h->cnorm;
  v->rowptr = h->rowptr;
  v->col = h->col;
  return true;
}

void* flr_aux_get(flr_t h) { return h ? h->aux : nullptr; }
void flr_aux_set(flr_t h, void* ws, void (*release)(void*)) {
  if (!h) return;
  h->aux = ws;
  h->aux_release = release;
}

extern "C" {

flr_status flr_get_info(flr_t h, int64_t* n, int64_t* p, int64_t* m, int32_t* dtype) {
  if (!h) return FLR_EINVAL;
  if (n) *n = h->n;
  if (p) *p = h->p;
  if (m) *m = h->m;
  if (dtype) *dtype = h->dtype;
  return FLR_OK;
}

}  // extern "C"
