// flr_solve_dense: Algorithm 1 of the paper on the GPU -- the MM iteration with
// each surrogate system (Eq. lin-sys)
//     Q(r) beta = X^T y,   Q(r) = X^T X + lam1 A(r) + lam2 B(r),
// solved by a dense Cholesky factorization instead of conjugate gradient.
// The paper recommends this route when E is a general graph (Section 4).
// Everything is FP64 on the CUDA cores:
//   - G = X^T X once per handle (tiled, X widened exactly from its storage type);
//   - per MM iteration: Q = G plus the diagonal lam1 a_j and the weighted
//     Laplacian entries, a right-looking blocked Cholesky Q = L L^T in 64 x 64
//     tiles (diagonal-tile factorization, panel triangular solve, trailing
//     update of the lower tiles), then L z = X^T y and L^T beta = z by blocked
//     substitution, then f(beta) from X beta;
//   - the host drives the loop and the stop test |f_new - f_old| / |f_old| <= tol.
// Matrices are column-major p x p; only the lower triangle of Q is referenced.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/flr.h"
#include "flr_internal.h"

namespace {

constexpr int NB = 64;       // tile order
constexpr int kDT = 256;     // threads of the tile kernels (16 x 16, 4 x 4 outputs each)

struct DenseWS {
  long long p = 0;
  double *G = nullptr, *Q = nullptr, *beta = nullptr, *z = nullptr, *red = nullptr;
  int* err = nullptr;
  bool gram_ready = false;
};

void ws_release(void* w) {
  DenseWS* d = static_cast<DenseWS*>(w);
  if (!d) return;
  cudaFree(d->G);
  cudaFree(d->Q);
  cudaFree(d->beta);
  cudaFree(d->z);
  cudaFree(d->red);
  cudaFree(d->err);
  delete d;
}

template <typename TX> __device__ __forceinline__ double wid(TX v);
template <> __device__ __forceinline__ double wid<double>(double v) { return v; }
template <> __device__ __forceinline__ double wid<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double wid<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <> __device__ __forceinline__ double wid<__half>(__half v) { return (double)__half2float(v); }

// lower-triangle tile (bi, bj), bi >= bj, of linear index t
__device__ __forceinline__ void tri_index(long long t, int& bi, int& bj) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(i + 1) * (i + 2) / 2 <= t) ++i;
  while ((long long)i * (i + 1) / 2 > t) --i;
  bi = i;
  bj = (int)(t - (long long)i * (i + 1) / 2);
}

// G = X^T X, both triangles (tile (bi, bj) and its mirror), FP64 accumulation
template <typename TX>
__global__ void __launch_bounds__(kDT) gram_kernel(const TX* __restrict__ Xt, long long n, long long p,
                                                   long long ldn, double* __restrict__ G) {
  __shared__ double A[32][NB + 1], B[32][NB + 1];
  int bi, bj;
  tri_index(blockIdx.x, bi, bj);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long long ci = (long long)bi * NB, cj = (long long)bj * NB;
  double acc[4][4] = {};
  for (long long i0 = 0; i0 < n; i0 += 32) {
    for (int e = threadIdx.x; e < 32 * NB; e += kDT) {
      const int ii = e & 31, col = e >> 5;
      const long long row = i0 + ii;
      A[ii][col] = (row < n && ci + col < p) ? wid<TX>(Xt[(ci + col) * ldn + row]) : 0.0;
      B[ii][col] = (row < n && cj + col < p) ? wid<TX>(Xt[(cj + col) * ldn + row]) : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < 32; ++ii)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(A[ii][ty * 4 + a], B[ii][tx * 4 + b], acc[a][b]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long long r = ci + ty * 4 + a, c = cj + tx * 4 + b;
      if (r < p && c < p) {
        G[c * p + r] = acc[a][b];
        G[r * p + c] = acc[a][b];
      }
    }
}

// Q += lam1 diag(a) + lam2 B from beta (Eq. lin-sys).  Thread j owns column j's
// diagonal and the lower entries (j, k), k < j, of its neighbours.
__global__ void assemble_kernel(double* __restrict__ Q, long long p, long long q2, const long long* rowptr,
                                const int* col, const double* __restrict__ beta, double lam1, double lam2,
                                double eps) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  const double bj = beta[j];
  double diag = lam1 / (fabs(bj) + eps);
  auto edge = [&](long long k) {
    const double w = lam2 / (fabs(bj - beta[k]) + eps);
    diag += w;
    if (k < j) Q[k * p + j] -= w;   // lower entry (row j, column k)
  };
  if (rowptr) {
    for (long long e = rowptr[j]; e < rowptr[j + 1]; ++e) edge(col[e]);
  } else {
    const long long cc = j % q2;
    if (cc != 0) edge(j - 1);
    if (cc != q2 - 1 && j + 1 < p) edge(j + 1);
    if (j >= q2) edge(j - q2);
    if (j + q2 < p) edge(j + q2);
  }
  Q[j * p + j] += diag;
}

// Cholesky of diagonal tile k in shared memory; a pivot <= 0 sets *err
__global__ void __launch_bounds__(kDT) potrf_tile(double* Q, long long p, int k, int* err) {
  __shared__ double T[NB][NB + 1];
  const long long o = (long long)k * NB;
  const int m = (int)(p - o < NB ? p - o : NB);
  for (int e = threadIdx.x; e < NB * NB; e += kDT) {
    const int r = e % NB, c = e / NB;
    T[r][c] = (r < m && c < m && r >= c) ? Q[(o + c) * p + (o + r)] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      double d = T[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicCAS(err, 0, 1);
        d = 1.0;
      }
      T[j][j] = sqrt(d);
    }
    __syncthreads();
    const double inv = 1.0 / T[j][j];
    for (int r = j + 1 + threadIdx.x; r < m; r += kDT) T[r][j] *= inv;
    __syncthreads();
    const int t = m - j - 1;   // trailing order
    for (int e = threadIdx.x; e < t * t; e += kDT) {
      const int r = j + 1 + e % t, c = j + 1 + e / t;
      if (r >= c) T[r][c] = fma(-T[r][j], T[c][j], T[r][c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NB * NB; e += kDT) {
    const int r = e % NB, c = e / NB;
    if (r < m && c < m && r >= c) Q[(o + c) * p + (o + r)] = T[r][c];
  }
}

// Panel: tile (i, k) := A_ik L_kk^-T for the row tiles i > k (one row per thread)
__global__ void __launch_bounds__(NB) trsm_tile(double* Q, long long p, int k) {
  __shared__ double L[NB][NB + 1], Am[NB][NB + 1];
  const int i = k + 1 + blockIdx.x;
  const long long ok = (long long)k * NB, oi = (long long)i * NB;
  const int mk = (int)(p - ok < NB ? p - ok : NB), mi = (int)(p - oi < NB ? p - oi : NB);
  for (int e = threadIdx.x; e < NB * NB; e += NB) {
    const int r = e % NB, c = e / NB;
    L[r][c] = (r < mk && c < mk && r >= c) ? Q[(ok + c) * p + (ok + r)] : 0.0;
    Am[r][c] = (r < mi && c < mk) ? Q[(ok + c) * p + (oi + r)] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x;
  if (r < mi) {
    for (int c = 0; c < mk; ++c) {
      double s = Am[r][c];
      for (int l = 0; l < c; ++l) s = fma(-Am[r][l], L[c][l], s);
      Am[r][c] = s / L[c][c];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += NB) {
    const int rr = e % NB, c = e / NB;
    if (rr < mi && c < mk) Q[(ok + c) * p + (oi + rr)] = Am[rr][c];
  }
}

// Trailing update: tile (i, j) -= L_ik L_jk^T for k < j <= i
__global__ void __launch_bounds__(kDT) update_tiles(double* Q, long long p, int k) {
  __shared__ double Ai[NB][NB + 1], Aj[NB][NB + 1];
  int ii, jj;
  tri_index(blockIdx.x, ii, jj);
  const int i = k + 1 + ii, j = k + 1 + jj;
  const long long ok = (long long)k * NB, oi = (long long)i * NB, oj = (long long)j * NB;
  for (int e = threadIdx.x; e < NB * NB; e += kDT) {
    const int r = e % NB, c = e / NB;
    const bool kc = ok + c < p;
    Ai[r][c] = (kc && oi + r < p) ? Q[(ok + c) * p + (oi + r)] : 0.0;
    Aj[r][c] = (kc && oj + r < p) ? Q[(ok + c) * p + (oj + r)] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
#pragma unroll 4
  for (int l = 0; l < NB; ++l)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(Ai[ty * 4 + a][l], Aj[tx * 4 + b][l], acc[a][b]);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long long r = oi + ty * 4 + a, c = oj + tx * 4 + b;
      if (r < p && c < p && r >= c) Q[c * p + r] -= acc[a][b];
    }
}

// Forward substitution on tile k: z_k := L_kk^-1 z_k (then the panel update)
__global__ void __launch_bounds__(NB) fsub_diag(const double* Q, long long p, int k, double* z) {
  __shared__ double zs[NB];
  const long long o = (long long)k * NB;
  const int m = (int)(p - o < NB ? p - o : NB);
  const int r = threadIdx.x;
  if (r < m) zs[r] = z[o + r];
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (r == j) zs[j] /= Q[(o + j) * p + (o + j)];
    __syncthreads();
    if (r > j && r < m) zs[r] = fma(-Q[(o + j) * p + (o + r)], zs[j], zs[r]);
    __syncthreads();
  }
  if (r < m) z[o + r] = zs[r];
}
// z_i -= L_ik z_k for the row tiles i > k (one row per thread)
__global__ void __launch_bounds__(NB) fsub_panel(const double* Q, long long p, int k, double* z) {
  const int i = k + 1 + blockIdx.x;
  const long long ok = (long long)k * NB, row = (long long)i * NB + threadIdx.x;
  const int mk = (int)(p - ok < NB ? p - ok : NB);
  if (row >= p) return;
  double s = 0.0;
  for (int c = 0; c < mk; ++c) s = fma(Q[(ok + c) * p + row], z[ok + c], s);
  z[row] -= s;
}
// Back substitution on tile k: b_k := L_kk^-T b_k
__global__ void __launch_bounds__(NB) bsub_diag(const double* Q, long long p, int k, double* b) {
  __shared__ double bs[NB];
  const long long o = (long long)k * NB;
  const int m = (int)(p - o < NB ? p - o : NB);
  const int r = threadIdx.x;
  if (r < m) bs[r] = b[o + r];
  __syncthreads();
  for (int j = m - 1; j >= 0; --j) {
    if (r == j) bs[j] /= Q[(o + j) * p + (o + j)];
    __syncthreads();
    if (r < j) bs[r] = fma(-Q[(o + r) * p + (o + j)], bs[j], bs[r]);
    __syncthreads();
  }
  if (r < m) b[o + r] = bs[r];
}
// b_i -= L_ki^T b_k for the row tiles i < k (one entry per thread)
__global__ void __launch_bounds__(NB) bsub_panel(const double* Q, long long p, int k, double* b) {
  const int i = blockIdx.x;
  const long long ok = (long long)k * NB, idx = (long long)i * NB + threadIdx.x;
  const int mk = (int)(p - ok < NB ? p - ok : NB);
  if (idx >= p) return;
  double s = 0.0;
  for (int c = 0; c < mk; ++c) s = fma(Q[idx * p + (ok + c)], b[ok + c], s);
  b[idx] -= s;
}

__global__ void init_kernel(const double* c, const double* d, long long p, double* beta) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < p) beta[j] = d[j] != 0.0 ? c[j] / d[j] : 0.0;
}

// red[0] += ||y - X beta||^2 (thread per row)
template <typename TX>
__global__ void rss_kernel(const TX* __restrict__ Xt, const double* __restrict__ y, long long n, long long p,
                           long long ldn, const double* __restrict__ beta, double* red) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    double u = 0.0;
    for (long long j = 0; j < p; ++j) u = fma(wid<TX>(Xt[j * ldn + i]), beta[j], u);
    const double r = y[i] - u;
    v = r * r;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(red, v);
}

// red[1] += sum |b_j|, red[2] += sum_E |b_j - b_k| (each edge once, from its
// lower end); red[3], red[4]: the same with p_eps(x) = |x| - eps log(1 + |x|/eps)
__global__ void penalty_kernel(long long p, long long q2, const long long* rowptr, const int* col,
                               const double* __restrict__ beta, double eps, double* red) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (j < p) {
    const double bj = beta[j];
    v[0] = fabs(bj);
    v[2] = fabs(bj) - eps * log1p(fabs(bj) / eps);
    auto up = [&](long long k) {
      const double dd = fabs(bj - beta[k]);
      v[1] += dd;
      v[3] += dd - eps * log1p(dd / eps);
    };
    if (rowptr) {
      for (long long e = rowptr[j]; e < rowptr[j + 1]; ++e)
        if (col[e] > j) up(col[e]);
    } else {
      if ((j % q2) != q2 - 1 && j + 1 < p) up(j + 1);
      if (j + q2 < p) up(j + q2);
    }
  }
  for (int f = 0; f < 4; ++f) {
    double s = v[f];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(red + 1 + f, s);
  }
}

struct Obj {
  double f, f_eps;
};

template <typename TX>
cudaError_t objective(const flr_view& v, DenseWS* w, double lam1, double lam2, double eps, Obj* out) {
  cudaError_t e = cudaMemsetAsync(w->red, 0, 8 * sizeof(double), v.stream);
  if (e != cudaSuccess) return e;
  rss_kernel<TX><<<(unsigned)((v.n + 255) / 256), 256, 0, v.stream>>>(static_cast<const TX*>(v.Xt), v.y, v.n,
                                                                    v.p, v.ldn, w->beta, w->red);
  penalty_kernel<<<(unsigned)((v.p + 255) / 256), 256, 0, v.stream>>>(
      v.p, v.q2, v.gkind == FLR_E_EDGES ? v.rowptr : nullptr, v.col, w->beta, eps, w->red);
  double h[8];
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, w->red, sizeof(h), cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess) return e;
  out->f = 0.5 * h[0] + lam1 * h[1] + lam2 * h[2];
  out->f_eps = 0.5 * h[0] + lam1 * h[3] + lam2 * h[4];
  return cudaSuccess;
}

template <typename TX>
cudaError_t gram(const flr_view& v, DenseWS* w) {
  const long long nt = (v.p + NB - 1) / NB;
  gram_kernel<TX><<<(unsigned)(nt * (nt + 1) / 2), kDT, 0, v.stream>>>(static_cast<const TX*>(v.Xt), v.n, v.p,
                                                                       v.ldn, w->G);
  return cudaGetLastError();
}

// one surrogate solve: Q = G + lam1 A + lam2 B, Q = L L^T, L L^T beta = X^T y
cudaError_t surrogate_solve(const flr_view& v, DenseWS* w, double lam1, double lam2, double eps, bool* spd) {
  const long long p = v.p, nt = (p + NB - 1) / NB;
  cudaStream_t st = v.stream;
  cudaError_t e = cudaMemcpyAsync(w->Q, w->G, sizeof(double) * p * p, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  assemble_kernel<<<(unsigned)((p + 255) / 256), 256, 0, st>>>(
      w->Q, p, v.q2, v.gkind == FLR_E_EDGES ? v.rowptr : nullptr, v.col, w->beta, lam1, lam2, eps);
  for (int k = 0; k < nt; ++k) {
    potrf_tile<<<1, kDT, 0, st>>>(w->Q, p, k, w->err);
    const long long rest = nt - k - 1;
    if (rest > 0) {
      trsm_tile<<<(unsigned)rest, NB, 0, st>>>(w->Q, p, k);
      update_tiles<<<(unsigned)(rest * (rest + 1) / 2), kDT, 0, st>>>(w->Q, p, k);
    }
  }
  e = cudaMemcpyAsync(w->z, v.c, sizeof(double) * p, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < nt; ++k) {
    fsub_diag<<<1, NB, 0, st>>>(w->Q, p, k, w->z);
    if (nt - k - 1 > 0) fsub_panel<<<(unsigned)(nt - k - 1), NB, 0, st>>>(w->Q, p, k, w->z);
  }
  for (int k = (int)nt - 1; k >= 0; --k) {
    bsub_diag<<<1, NB, 0, st>>>(w->Q, p, k, w->z);
    if (k > 0) bsub_panel<<<(unsigned)k, NB, 0, st>>>(w->Q, p, k, w->z);
  }
  int herr = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, w->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *spd = herr == 0;
  if (*spd) e = cudaMemcpyAsync(w->beta, w->z, sizeof(double) * p, cudaMemcpyDeviceToDevice, st);
  return e;
}

template <typename TX>
flr_status run_dense(const flr_view& v, DenseWS* w, double lam1, double lam2, double eps, double tol,
                     int max_mm, const double* beta_init, int io_mem, flr_stats* stats, double* beta_out) {
  cudaStream_t st = v.stream;
  auto fail = [](cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FLR_ENOMEM : FLR_ECUDA;
  };
  cudaError_t e = cudaSuccess;
  if (!w->gram_ready) {
    if ((e = gram<TX>(v, w)) != cudaSuccess) return fail(e);
    w->gram_ready = true;
  }
  if (beta_init) {
    e = cudaMemcpyAsync(w->beta, beta_init, sizeof(double) * v.p,
                        io_mem == FLR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
  } else {
    init_kernel<<<(unsigned)((v.p + 255) / 256), 256, 0, st>>>(v.c, v.d, v.p, w->beta);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(e);
  Obj ob{};
  if ((e = objective<TX>(v, w, lam1, lam2, eps, &ob)) != cudaSuccess) return fail(e);
  flr_status status = FLR_OK;
  double rel = 0.0;
  int mm = 0;
  while (true) {
    if (!std::isfinite(ob.f)) { status = FLR_ENONFINITE; break; }
    if (mm >= max_mm) { status = FLR_ENOTCONV; break; }
    bool spd = true;
    if ((e = surrogate_solve(v, w, lam1, lam2, eps, &spd)) != cudaSuccess) return fail(e);
    if (!spd) { status = FLR_EBREAKDOWN; break; }
    ++mm;
    Obj nb{};
    if ((e = objective<TX>(v, w, lam1, lam2, eps, &nb)) != cudaSuccess) return fail(e);
    rel = std::fabs(nb.f - ob.f) / std::fabs(ob.f);
    ob = nb;
    if (rel <= tol) break;
  }
  e = cudaMemcpyAsync(beta_out, w->beta, sizeof(double) * v.p,
                      io_mem == FLR_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  if (stats) {
    stats->mm_iters = mm;
    stats->cg_iters = 0;
    stats->status = status;
    stats->f = ob.f;
    stats->f_eps = ob.f_eps;
    stats->rel_change = rel;
    stats->cg_relres = 0.0;
    stats->refine_steps = 0;
    stats->reserved = 0;
    const double gap = std::fabs(ob.f) > 0 ? (ob.f - ob.f_eps) / std::fabs(ob.f) : 0.0;
    stats->est_err = std::max(0.0, gap) + rel;
  }
  return status;
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
    (void)cudaGetLastError();
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" flr_status flr_solve_dense(flr_t h, double lambda1, double lambda2, double eps, double tol,
                                      int32_t max_mm, const double* beta_init, double* beta_out,
                                      int32_t io_mem, flr_stats* stats) {
  flr_view v{};
  if (!flr_get_view(h, &v) || !beta_out) return FLR_EINVAL;
  if (!(lambda1 >= 0.0) || !(lambda2 >= 0.0) || !(eps > 0.0) || !(tol > 0.0) || max_mm < 0) return FLR_EINVAL;
  if (!std::isfinite(lambda1) || !std::isfinite(lambda2) || !std::isfinite(eps)) return FLR_EINVAL;
  if (io_mem != FLR_MEM_DEVICE && io_mem != FLR_MEM_HOST) return FLR_EINVAL;
  if (v.dtype == FLR_IDENTITY) return FLR_ENOTIMPL;
  if (v.p > FLR_DENSE_MAX_P) return FLR_ENOTIMPL;
  DevGuard dg(v.device);
  const auto t0 = std::chrono::steady_clock::now();
  DenseWS* w = static_cast<DenseWS*>(flr_aux_get(h));
  if (!w) {
    w = new (std::nothrow) DenseWS();
    if (!w) return FLR_ENOMEM;
    const long long p = v.p;
    w->p = p;
    cudaError_t e = cudaMalloc(&w->G, sizeof(double) * p * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->Q, sizeof(double) * p * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->beta, sizeof(double) * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->z, sizeof(double) * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->red, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&w->err, sizeof(int));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      ws_release(w);
      return FLR_ENOMEM;
    }
    flr_aux_set(h, w, ws_release);
  }
  flr_status s;
  switch (v.dtype) {
    case FLR_F64: s = run_dense<double>(v, w, lambda1, lambda2, eps, tol, max_mm, beta_init, io_mem, stats, beta_out); break;
    case FLR_F32: s = run_dense<float>(v, w, lambda1, lambda2, eps, tol, max_mm, beta_init, io_mem, stats, beta_out); break;
    case FLR_BF16: s = run_dense<__nv_bfloat16>(v, w, lambda1, lambda2, eps, tol, max_mm, beta_init, io_mem, stats, beta_out); break;
    case FLR_F16: s = run_dense<__half>(v, w, lambda1, lambda2, eps, tol, max_mm, beta_init, io_mem, stats, beta_out); break;
    default: return FLR_EINVAL;
  }
  if (stats) {
    stats->grid = 0;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return s;
}
