// The MM solve of fused lasso regression as one persistent cooperative kernel.
//
// Method (Section 3): MM iteration r reweights
//     a_j = 1/(|b_j| + eps),  w_jk = 1/(|b_j - b_k| + eps)           (Eq. lin-sys)
// from the iterate b = beta(r) and solves
//     Q b' = c,  Q = X^T X + lam1 A + lam2 B,  c = X^T y              (Eq. lin-sys)
// by preconditioned CG warm-started at x0 = beta(r) (Algorithm 2), then
// stops when |f(beta(r+1)) - f(beta(r))| / |f(beta(r))| <= tol.
//
// Work decomposition: block b owns the contiguous coefficient range
// [j0, j1) and the matching column slab of X, stored column-major (Xt[j][i]
// = X[i][j], row length ldn).  One CG iteration is
//   phase A: u += X[:, j0:j1] p[j0:j1]   (FP32 or FP64 atomics into u)
//            Sp_j = lam1 a_j p_j + lam2 sum_k w_jk (p_j - p_k) and p^T S p
//   barrier 1
//            p^T Q p = ||u||^2 + p^T S p;  nu = r^T z / p^T Q p
//   phase C: t_j = X[:, j]^T u;  q = t + Sp;  x += nu p;  r -= nu q
//            z = M^-1 r;  partial r^T z, r^T r
//   barrier 2
//            gamma = r^T z / (r^T z)_old;  p = z + gamma p
// The residual update uses r_j = r_{j-1} - nu Q p (the sign that keeps
// r = c - Q x; Algorithm 2 prints "+").  Every scalar reduction sums
// per-block partials in a fixed order, so all blocks take identical
// decisions.  Halo values of p (neighbours owned by other blocks) are
// recomputed as z_k + gamma p_old_k from double-buffered p, bit-identical
// to the owner's own update.
#pragma once
#include "flr_device.cuh"

namespace flr {

struct DevStats {
  int mm_iters, cg_iters, status, pad;
  double f, f_eps, rel_change, cg_relres;
};

enum PrecondKind : int { PC_JACOBI = 1, PC_TRIDIAG = 2, PC_PAPER = 3 };
enum GraphKind : int { GK_STENCIL = 0, GK_CSR = 1 };
enum SolveStatus : int {
  ST_OK = 0, ST_NOTCONV = 4, ST_BREAKDOWN = 5, ST_NONFINITE = 6, ST_TIMEOUT = 7
};

struct SolveParams {
  const void* Xt;
  long long n, p, ldn;
  const double* y;
  const double* c;
  const double* d;
  double cnorm;
  long long q2;              // stencil row length (chain: p)
  const long long* rowptr;   // CSR (both orientations of every edge)
  const int* col;
  double lam1, lam2, eps, tol, tol_cg;
  int max_mm, max_cg, min_cg, precond;
  long long w, wpad;         // coefficients per block, padded to a multiple of 4
  int levels;                // PCR levels for the block chunk
  const double* beta_init;   // nullptr -> X_j^T y / X_j^T X_j
  // state
  double *x, *r, *z, *pb0, *pb1, *q, *a, *wL, *wR, *wU, *wD, *wc, *idg, *K1, *K2, *binv;
  void* ub0;
  void* ub1;
  double* part;              // [2 slots][kNF][gridDim.x]
  unsigned* bar;
  int* err;
  DevStats* stats;
  long long timeout;
  int inject_stall;          // test hook: block 0 skips the first barrier
};

// u[0:n] += sum_{j in slab} X[:, j] * v[j - j0]   (v staged in shared memory)
template <typename TX>
__device__ __forceinline__ void phase_a(const SolveParams& P, const TX* __restrict__ Xt,
                                        long long j0, int wl,
                                        const typename XT<TX>::Acc* vs,
                                        typename XT<TX>::Acc* red,
                                        typename XT<TX>::Acc* u) {
  using Acc = typename XT<TX>::Acc;
  constexpr int V = XT<TX>::V;
  const int tid = threadIdx.x;
  const long long nv = P.ldn / V;
  if (wl <= 0) return;
  if (nv >= kThreads) {
    for (long long rv = tid; rv < nv; rv += kThreads) {
      Acc acc[V];
#pragma unroll
      for (int e = 0; e < V; ++e) acc[e] = Acc(0);
      const TX* base = Xt + j0 * P.ldn + rv * V;
      int j = 0;
      for (; j + 4 <= wl; j += 4) {
        uint4 raw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) raw[k] = ld_stream16(base + (long long)(j + k) * P.ldn);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Acc xv[V];
          XT<TX>::cvt(raw[k], xv);
          const Acc s = vs[j + k];
#pragma unroll
          for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
        }
      }
      for (; j < wl; ++j) {
        Acc xv[V];
        XT<TX>::cvt(ld_stream16(base + (long long)j * P.ldn), xv);
        const Acc s = vs[j];
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
      }
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const long long i = rv * V + e;
        if (i < P.n && acc[e] != Acc(0)) atomicAdd(u + i, acc[e]);
      }
    }
  } else {
    const int ncg = kThreads / (int)nv;          // column groups, >= 1
    const int rv = tid % (int)nv, cg = tid / (int)nv;
    Acc acc[V];
#pragma unroll
    for (int e = 0; e < V; ++e) acc[e] = Acc(0);
    if (cg < ncg) {
      const TX* base = Xt + j0 * P.ldn + (long long)rv * V;
      int j = cg;
      for (; j + 3 * ncg < wl; j += 4 * ncg) {
        uint4 raw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) raw[k] = ld_stream16(base + (long long)(j + k * ncg) * P.ldn);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Acc xv[V];
          XT<TX>::cvt(raw[k], xv);
          const Acc s = vs[j + k * ncg];
#pragma unroll
          for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
        }
      }
      for (; j < wl; j += ncg) {
        Acc xv[V];
        XT<TX>::cvt(ld_stream16(base + (long long)j * P.ldn), xv);
        const Acc s = vs[j];
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
      }
#pragma unroll
      for (int e = 0; e < V; ++e) red[(long long)cg * nv * V + (long long)rv * V + e] = acc[e];
    }
    __syncthreads();
    const int rows = (int)nv * V;
    for (int i = tid; i < rows; i += kThreads) {
      Acc s = Acc(0);
      for (int g = 0; g < ncg; ++g) s += red[g * rows + i];
      if (i < P.n && s != Acc(0)) atomicAdd(u + i, s);
    }
    __syncthreads();
  }
}

// tv[jj] = X[:, j0+jj]^T u  for jj in [0, wl)   (u staged in shared memory)
template <typename TX>
__device__ __forceinline__ void phase_c(const SolveParams& P, const TX* __restrict__ Xt,
                                        long long j0, int wl,
                                        const typename XT<TX>::Acc* us, double* tv) {
  using Acc = typename XT<TX>::Acc;
  constexpr int V = XT<TX>::V;
  constexpr int CPW = 4;  // columns per warp in flight
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = (int)(P.ldn / V);
  for (int base = warp * CPW; base < wl; base += kWarps * CPW) {
    Acc acc[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) acc[c] = Acc(0);
    for (int rv = lane; rv < nv; rv += 32) {
      Acc uu[V];
#pragma unroll
      for (int e = 0; e < V; ++e) uu[e] = us[rv * V + e];
      uint4 raw[CPW];
#pragma unroll
      for (int c = 0; c < CPW; ++c)
        if (base + c < wl) raw[c] = ld_stream16(Xt + (j0 + base + c) * P.ldn + (long long)rv * V);
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        if (base + c < wl) {
          Acc xv[V];
          XT<TX>::cvt(raw[c], xv);
#pragma unroll
          for (int e = 0; e < V; ++e) acc[c] = fma(xv[e], uu[e], acc[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const Acc s = warp_sum(acc[c]);
      if (lane == 0 && base + c < wl) tv[base + c] = (double)s;
    }
  }
  __syncthreads();
}

// z[own] = M^-1 r[own].  Jacobi: r * idg.  Tridiagonal: parallel cyclic
// reduction over the block's chunk with multipliers precomputed per MM
// iteration (K1, K2, binv); `w0`/`w1` are two chunk-sized shared buffers.
__device__ __forceinline__ void apply_precond(const SolveParams& P, long long j0, int wl,
                                              double* w0, double* w1) {
  const int tid = threadIdx.x;
  if (P.precond == PC_JACOBI) {
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      P.z[j] = P.r[j] * P.idg[j];
    }
    __syncthreads();
    return;
  }
  for (int jj = tid; jj < wl; jj += kThreads) w0[jj] = P.r[j0 + jj];
  __syncthreads();
  double* cur = w0;
  double* nxt = w1;
  for (int l = 0; l < P.levels; ++l) {
    const int s = 1 << l;
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      double v = cur[jj];
      if (jj >= s) v = fma(-P.K1[(long long)l * P.p + j], cur[jj - s], v);
      if (jj + s < wl) v = fma(-P.K2[(long long)l * P.p + j], cur[jj + s], v);
      nxt[jj] = v;
    }
    __syncthreads();
    double* t = cur; cur = nxt; nxt = t;
  }
  for (int jj = tid; jj < wl; jj += kThreads) P.z[j0 + jj] = cur[jj] * P.binv[j0 + jj];
  __syncthreads();
}

// Precompute the PCR multipliers of the chunk's tridiagonal matrix
// (diag D, couplings -lam2 w between consecutive indices inside the chunk).
__device__ __forceinline__ void setup_tridiag(const SolveParams& P, long long j0, int wl,
                                              double* sm6) {
  const int tid = threadIdx.x;
  const long long wp = P.wpad;
  double* A0 = sm6;          double* B0 = sm6 + wp;     double* C0 = sm6 + 2 * wp;
  double* A1 = sm6 + 3 * wp; double* B1 = sm6 + 4 * wp; double* C1 = sm6 + 5 * wp;
  for (int jj = tid; jj < wl; jj += kThreads) {
    const long long j = j0 + jj;
    double dj = P.lam1 * P.a[j];
    // full weighted degree on the diagonal (all edges of j)
    double deg = P.wL[j] + P.wR[j] + P.wU[j] + P.wD[j];
    dj = fma(P.lam2, deg, dj);
    if (P.precond == PC_TRIDIAG) dj += P.d[j];
    B0[jj] = dj;
    A0[jj] = jj > 0 ? -P.lam2 * P.wL[j] : 0.0;
    C0[jj] = jj + 1 < wl ? -P.lam2 * P.wR[j] : 0.0;
  }
  __syncthreads();
  double *A = A0, *B = B0, *C = C0, *An = A1, *Bn = B1, *Cn = C1;
  for (int l = 0; l < P.levels; ++l) {
    const int s = 1 << l;
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      double k1 = 0.0, k2 = 0.0, b = B[jj], an = 0.0, cn = 0.0;
      if (jj >= s) {
        k1 = A[jj] / B[jj - s];
        an = -A[jj - s] * k1;
        b = fma(-C[jj - s], k1, b);
      }
      if (jj + s < wl) {
        k2 = C[jj] / B[jj + s];
        cn = -C[jj + s] * k2;
        b = fma(-A[jj + s], k2, b);
      }
      P.K1[(long long)l * P.p + j] = k1;
      P.K2[(long long)l * P.p + j] = k2;
      An[jj] = an; Bn[jj] = b; Cn[jj] = cn;
    }
    __syncthreads();
    double* t;
    t = A; A = An; An = t;
    t = B; B = Bn; Bn = t;
    t = C; C = Cn; Cn = t;
  }
  for (int jj = tid; jj < wl; jj += kThreads) P.binv[j0 + jj] = 1.0 / B[jj];
  __syncthreads();
}

__device__ __forceinline__ double edge_w(double xj, double xk, double eps) {
  return 1.0 / (fabs(xj - xk) + eps);
}

template <typename TX, int GK>
__global__ void __launch_bounds__(kThreads, 1) mm_solve_kernel(const SolveParams P) {
  using Acc = typename XT<TX>::Acc;
  constexpr int V = XT<TX>::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tid = threadIdx.x;
  const int G = gridDim.x, b = blockIdx.x;
  const long long p = P.p, n = P.n, q2 = P.q2;
  const long long j0 = (long long)b * P.w;
  const long long j1 = j0 + P.w < p ? j0 + P.w : p;
  const int wl = j1 > j0 ? (int)(j1 - j0) : 0;
  const int nwc = wl >= kThreads ? kWarps : (wl + 31) / 32;          // warps with column data
  const int nwn = n >= kThreads ? kWarps : (int)((n + 31) / 32);    // warps with row data
  const int nwg = (G + 31) / 32;

  Acc* us = reinterpret_cast<Acc*>(smraw);
  Acc* vs = us + P.ldn;
  Acc* red = vs + P.wpad;
  double* tv = reinterpret_cast<double*>(red + kThreads * V);
  double* pw = tv + P.wpad;          // 6 * wpad doubles (PCR)
  double* rs = pw + 6 * P.wpad;      // kWarps*kNF + kNF doubles
  const TX* Xt = reinterpret_cast<const TX*>(P.Xt);
  Acc* ub[2] = {reinterpret_cast<Acc*>(P.ub0), reinterpret_cast<Acc*>(P.ub1)};
  double* pbuf[2] = {P.pb0, P.pb1};
  GridBarrier gb{P.bar, P.err, 0u, P.timeout};
  int slot = 0;

  // grid-wide sum of kNF fields (each block contributes v, all blocks get totals)
  auto grid_sum = [&](double (&v)[kNF]) -> bool {
    if (tid == 0) {
#pragma unroll
      for (int f = 0; f < kNF; ++f) P.part[((long long)slot * kNF + f) * G + b] = v[f];
    }
    if (!gb.sync()) return false;
#pragma unroll
    for (int f = 0; f < kNF; ++f)
      v[f] = tid < G ? ldcg(&P.part[((long long)slot * kNF + f) * G + tid]) : 0.0;
    block_sum<kNF>(v, rs, nwg);
    slot ^= 1;
    return true;
  };

  // ---- initialisation (Algorithm 1): beta_j = X_j^T y / X_j^T X_j
  for (int jj = tid; jj < wl; jj += kThreads) {
    const long long j = j0 + jj;
    double v;
    if (P.beta_init) v = P.beta_init[j];
    else v = P.d[j] != 0.0 ? P.c[j] / P.d[j] : 0.0;
    P.x[j] = v;
  }
  if (P.inject_stall && b == 0) return;   // the others' bounded waits must expire
  if (!gb.sync()) return;

  int cur_u = 0, pcur = 0, mm = 0, cg_total = 0, status = ST_OK;
  double f = 0.0, f_prev = 0.0, rel = 0.0, relres = 0.0, rss_last = 0.0;

  while (true) {
    // ---------------- reweight (Eq. lin-sys) and S x for the CG start
    double loc[kNF] = {0.0, 0.0, 0.0, 0.0};   // sum|x_j|, sum_E|x_j - x_k|
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      const double xj = ldcg(P.x + j);
      const double aj = 1.0 / (fabs(xj) + P.eps);
      P.a[j] = aj;
      double deg = 0.0, lap = 0.0;
      if (GK == GK_STENCIL) {
        const long long col = j % q2;
        double wl_ = 0.0, wr_ = 0.0, wu_ = 0.0, wd_ = 0.0;
        if (col != 0) {
          const double xk = ldcg(P.x + j - 1);
          wl_ = edge_w(xk, xj, P.eps);
          lap = fma(wl_, xj - xk, lap);
        }
        if (col != q2 - 1 && j + 1 < p) {
          const double xk = ldcg(P.x + j + 1);
          wr_ = edge_w(xj, xk, P.eps);
          lap = fma(wr_, xj - xk, lap);
          loc[1] += fabs(xj - xk);
        }
        if (j >= q2) {
          const double xk = ldcg(P.x + j - q2);
          wu_ = edge_w(xk, xj, P.eps);
          lap = fma(wu_, xj - xk, lap);
        }
        if (j + q2 < p) {
          const double xk = ldcg(P.x + j + q2);
          wd_ = edge_w(xj, xk, P.eps);
          lap = fma(wd_, xj - xk, lap);
          loc[1] += fabs(xj - xk);
        }
        P.wL[j] = wl_; P.wR[j] = wr_; P.wU[j] = wu_; P.wD[j] = wd_;
        deg = (wl_ + wr_) + (wu_ + wd_);
      } else {
        for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e) {
          const long long k = P.col[e];
          const double xk = ldcg(P.x + k);
          const double we = k > j ? edge_w(xj, xk, P.eps) : edge_w(xk, xj, P.eps);
          P.wc[e] = we;
          deg += we;
          lap = fma(we, xj - xk, lap);
          if (k > j) loc[1] += fabs(xj - xk);
        }
      }
      loc[0] += fabs(xj);
      const double dq = fma(P.lam2, deg, fma(P.lam1, aj, P.d[j]));
      P.idg[j] = 1.0 / dq;
      P.q[j] = fma(P.lam1 * aj, xj, P.lam2 * lap);      // (lam1 A + lam2 B) x
      vs[jj] = (Acc)xj;
    }
    if (P.precond != PC_JACOBI && GK == GK_STENCIL) {
      __syncthreads();
      setup_tridiag(P, j0, wl, pw);
    }
    __syncthreads();
    // ---------------- u0 = X x (for f and for r0)
    {
      const long long zs = (long long)b * ((n + G - 1) / G);
      const long long ze = zs + (n + G - 1) / G < n ? zs + (n + G - 1) / G : n;
      for (long long i = zs + tid; i < ze; i += kThreads) ub[cur_u ^ 1][i] = Acc(0);
    }
    phase_a<TX>(P, Xt, j0, wl, vs, red, ub[cur_u]);
    block_sum<kNF>(loc, rs, nwc);
    if (!grid_sum(loc)) return;
    // ---------------- objective f(beta(r)) (Eq. obj) and outer stop
    {
      double rv[kNF] = {0.0, 0.0, 0.0, 0.0};
      const Acc* u = ub[cur_u];
      for (long long i = tid; i < n; i += kThreads) {
        const Acc ui = ldcg(u + i);
        us[i] = ui;
        const double e = P.y[i] - (double)ui;
        rv[0] = fma(e, e, rv[0]);
      }
      for (long long i = n + tid; i < P.ldn; i += kThreads) us[i] = Acc(0);
      block_sum<kNF>(rv, rs, nwn);
      rss_last = rv[0];
      f = 0.5 * rv[0] + P.lam1 * loc[0] + P.lam2 * loc[1];
    }
    if (!isfinite(f)) { status = ST_NONFINITE; break; }
    if (mm > 0) {
      rel = fabs(f - f_prev) / fabs(f_prev);
      if (rel <= P.tol) break;
    }
    if (mm >= P.max_mm) { status = ST_NOTCONV; break; }
    // ---------------- r0 = c - Q x0, z0 = M^-1 r0, p1 = z0 (Algorithm 2)
    phase_c<TX>(P, Xt, j0, wl, us, tv);
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      P.r[j] = P.c[j] - tv[jj] - P.q[j];
    }
    __syncthreads();
    apply_precond(P, j0, wl, pw, pw + P.wpad);
    double rzv[kNF] = {0.0, 0.0, 0.0, 0.0};
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      const double rj = P.r[j], zj = P.z[j];
      pbuf[pcur][j] = zj;
      rzv[0] = fma(rj, zj, rzv[0]);
      rzv[1] = fma(rj, rj, rzv[1]);
    }
    block_sum<kNF>(rzv, rs, nwc);
    if (!grid_sum(rzv)) return;
    double rz = rzv[0], rr = rzv[1], gamma = 0.0;
    cur_u ^= 1;
    // ---------------- CG iterations
    int k = 0;
    while (true) {
      relres = sqrt(rr) / P.cnorm;
      if (k >= P.max_cg || (k >= P.min_cg && relres <= P.tol_cg)) break;
      const double* pc = pbuf[pcur];
      const double* po = pbuf[pcur ^ 1];
      // S p with halo p recomputed from (z, p_old) for k > 0
      double sv[kNF] = {0.0, 0.0, 0.0, 0.0};
      auto pval = [&](long long kk) -> double {
        if (kk >= j0 && kk < j1) return pc[kk];
        if (k == 0) return ldcg(pc + kk);
        return fma(gamma, ldcg(po + kk), ldcg(P.z + kk));
      };
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        const double pj = pc[j];
        double lap = 0.0;
        if (GK == GK_STENCIL) {
          const long long col = j % q2;
          if (col != 0) lap = fma(P.wL[j], pj - pval(j - 1), lap);
          if (col != q2 - 1 && j + 1 < p) lap = fma(P.wR[j], pj - pval(j + 1), lap);
          if (j >= q2) lap = fma(P.wU[j], pj - pval(j - q2), lap);
          if (j + q2 < p) lap = fma(P.wD[j], pj - pval(j + q2), lap);
        } else {
          for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e)
            lap = fma(P.wc[e], pj - pval(P.col[e]), lap);
        }
        const double spj = fma(P.lam1 * P.a[j], pj, P.lam2 * lap);
        P.q[j] = spj;
        sv[0] = fma(pj, spj, sv[0]);
        vs[jj] = (Acc)pj;
      }
      {
        const long long zs = (long long)b * ((n + G - 1) / G);
        const long long ze = zs + (n + G - 1) / G < n ? zs + (n + G - 1) / G : n;
        for (long long i = zs + tid; i < ze; i += kThreads) ub[cur_u ^ 1][i] = Acc(0);
      }
      __syncthreads();
      phase_a<TX>(P, Xt, j0, wl, vs, red, ub[cur_u]);
      block_sum<kNF>(sv, rs, nwc);
      if (!grid_sum(sv)) return;
      // p^T Q p = ||X p||^2 + p^T S p
      double uu[kNF] = {0.0, 0.0, 0.0, 0.0};
      {
        const Acc* u = ub[cur_u];
        for (long long i = tid; i < n; i += kThreads) {
          const Acc ui = ldcg(u + i);
          us[i] = ui;
          uu[0] = fma((double)ui, (double)ui, uu[0]);
        }
        block_sum<kNF>(uu, rs, nwn);
      }
      const double pq = uu[0] + sv[0];
      if (!(pq > 0.0) || !isfinite(pq)) { status = isfinite(pq) ? ST_BREAKDOWN : ST_NONFINITE; break; }
      const double nu = rz / pq;
      phase_c<TX>(P, Xt, j0, wl, us, tv);
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        const double pj = pc[j];
        const double qj = tv[jj] + P.q[j];
        P.x[j] = fma(nu, pj, P.x[j]);
        P.r[j] = fma(-nu, qj, P.r[j]);
      }
      __syncthreads();
      apply_precond(P, j0, wl, pw, pw + P.wpad);
      double rzn[kNF] = {0.0, 0.0, 0.0, 0.0};
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        const double rj = P.r[j];
        rzn[0] = fma(rj, P.z[j], rzn[0]);
        rzn[1] = fma(rj, rj, rzn[1]);
      }
      block_sum<kNF>(rzn, rs, nwc);
      if (!grid_sum(rzn)) return;
      gamma = rzn[0] / rz;
      rz = rzn[0];
      rr = rzn[1];
      // p_{j+1} = z_j + gamma p_j into the other buffer
      double* pn = pbuf[pcur ^ 1];
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        pn[j] = fma(gamma, pc[j], P.z[j]);
      }
      pcur ^= 1;
      cur_u ^= 1;
      ++k;
      __syncthreads();
    }
    cg_total += k;
    if (status != ST_OK) break;
    f_prev = f;
    ++mm;
    // x was written before the last grid barrier (or is unchanged): the next
    // reweight may read neighbours' x directly.
    if (k == 0 && !gb.sync()) return;
  }

  // ---------------- f_eps at the returned iterate (Eq. pert)
  {
    double loc[kNF] = {0.0, 0.0, 0.0, 0.0};
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      const double xj = ldcg(P.x + j);
      const double ax = fabs(xj);
      loc[0] += ax - P.eps * log1p(ax / P.eps);
      if (GK == GK_STENCIL) {
        const long long col = j % q2;
        if (col != q2 - 1 && j + 1 < p) {
          const double dd = fabs(xj - ldcg(P.x + j + 1));
          loc[1] += dd - P.eps * log1p(dd / P.eps);
        }
        if (j + q2 < p) {
          const double dd = fabs(xj - ldcg(P.x + j + q2));
          loc[1] += dd - P.eps * log1p(dd / P.eps);
        }
      } else {
        for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e) {
          const long long k = P.col[e];
          if (k > j) {
            const double dd = fabs(xj - ldcg(P.x + k));
            loc[1] += dd - P.eps * log1p(dd / P.eps);
          }
        }
      }
    }
    block_sum<kNF>(loc, rs, nwc);
    if (!grid_sum(loc)) return;
    if (b == 0 && tid == 0) {
      DevStats* S = P.stats;
      S->mm_iters = mm;
      S->cg_iters = cg_total;
      S->status = status;
      S->pad = 0;
      S->f = f;
      S->f_eps = 0.5 * rss_last + P.lam1 * loc[0] + P.lam2 * loc[1];
      S->rel_change = rel;
      S->cg_relres = relres;
    }
  }
}

}  // namespace flr
