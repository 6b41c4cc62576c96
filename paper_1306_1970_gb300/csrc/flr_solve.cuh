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
// = X[i][j], row length ldn).
//
// Once per MM iteration (refinement pass, FP64 accumulation over exactly
// widened X): u0 = X b, f(b) from u0 (Eq. obj), r0 = c - X^T u0 - S b with
// S = lam1 A + lam2 B.  This is the outer residual of a mixed-precision
// iterative refinement: the inner CG below may use FP32 products, while
// every MM iteration restarts from an FP64-accurate residual and objective.
// With max_refine > 0 the same is done inside an MM iteration: after the CG
// meets tol_cg on its recursive residual, the true residual of the same
// surrogate system is recomputed in FP64 and CG restarts from it until that
// residual meets tol_cg too (at most max_refine times), so each surrogate is
// solved to FP64 accuracy and the iterates follow the exact MM map.
//
// One CG iteration (products accumulate in FP32 for FP32/BF16/FP16 X):
//   phase A: u += X[:, j0:j1] p[j0:j1]   (atomics into u)
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
//
// Two-level preconditioner (PC_TWOLEVEL).  Fused neighbours (|b_j - b_k|
// near 0) couple with lam2 w_jk ~ lam2 / eps, far above d_j + lam1 a_j, and
// every connected group of such strong couplings leaves Q with a tiny
// eigenvalue along the group's constant vector, which Jacobi does not see.
// The preconditioner adds a coarse correction on exactly those directions:
//   M^-1 r = D^-1 r + sum_c 1_c (1_c^T r) / q_c,
// D = diag(Q), or on a chain the chunk-tridiagonal part of Q (TRIDIAG),
//   q_c = sum_{j in c} (d_j + lam1 a_j) + sum of lam2 w_e over edges e
//         leaving c,
// i.e. the diagonal of P^T Q P for the piecewise-constant P of the groups,
// with ||X 1_c||^2 replaced by sum_{j in c} d_j.  M^-1 is SPD for any
// partition.  An edge is strong when lam2 w_jk >= kStrong * min(d_j +
// lam1 a_j, d_k + lam1 a_k); the groups (components of size >= 2 of the
// strong edges) come from a lock-free union-find, once per MM iteration.
// Per CG iteration the component sums 1_c^T r are accumulated by atomics
// before barrier 2, and every block adds sum_c (1_c^T r)^2 / q_c to r^T z
// itself after it, so the CG iteration keeps two grid barriers.
//
// FP64 arithmetic is scarce on this GPU, so scalar work runs in one thread
// and block reductions go through shared memory and a single warp.
#pragma once
#include <cmath>
#include <type_traits>

#include "flr_device.cuh"
#include "flr_tc.cuh"

namespace flr {

struct DevStats {
  int mm_iters, cg_iters, status, refine_steps;
  double f, f_eps, rel_change, cg_relres;
  double rel_prev;           // the relative change of f one MM iteration earlier
  unsigned long long t0_ns, t1_ns;   // device global timer at the kernel's start and end
};

enum PrecondKind : int { PC_JACOBI = 1, PC_TRIDIAG = 2, PC_PAPER = 3, PC_TWOLEVEL = 4 };
enum GraphKind : int { GK_STENCIL = 0, GK_CSR = 1 };
enum SolveStatus : int {
  ST_OK = 0, ST_NOTCONV = 4, ST_BREAKDOWN = 5, ST_NONFINITE = 6, ST_TIMEOUT = 7
};
// neighbour flags of a coefficient; the high bits mark strong edges (PC_TWOLEVEL;
// edge lists use NB_SR for "has a strong edge")
enum NbrBits : unsigned char {
  NB_L = 1, NB_R = 2, NB_U = 4, NB_D = 8, NB_SL = 16, NB_SR = 32, NB_SU = 64, NB_SD = 128
};
constexpr unsigned char NB_STRONG = NB_SL | NB_SR | NB_SU | NB_SD;
constexpr double kStrong = 16.0;   // strong-edge threshold of PC_TWOLEVEL

constexpr int kRF = 3;   // fields per block reduction
constexpr int kLA = 16;  // 16-byte X loads in flight per thread in phase A
// One-pass (chunked) Q-apply (x_smem = 1): row chunks of kCRV 16-byte
// row vectors, kCCG column groups.
constexpr int kCRV = 16;
constexpr int kCCG = kThreads / kCRV;
constexpr int kLC = 8;    // loads in flight per thread in the chunked phase A
constexpr int kLCC = 8;   // and in the chunked phase C (a power of two <= kCRV)

constexpr int kUR = 1;   // replicas of each u accumulator: block b adds into replica b % kUR,
                         // spreading the atomics of X p over kUR times more L2 lines

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
  double tol_cg_rel;         // adaptive inner tolerance factor (0 = off)
  int max_mm, max_cg, min_cg, precond;
  int max_refine;            // FP64 residual restarts of the inner solve per MM iteration
  int ws;                    // slab columns kept in shared memory (after the TMEM ones)
  int wt;                    // leading slab columns kept in TMEM (0 = none)
  int tct;                   // TMEM cells per 128-row group (0 = no TMEM)
  int chunked;               // one-pass chunked Q-apply (x_smem = 1)
  unsigned* cbar;            // its two split-barrier counters (128 bytes apart)
  long long w, wpad;         // coefficients per block, padded to a multiple of 4
  int levels;                // PCR levels for the block chunk
  const double* beta_init;   // nullptr -> X_j^T y / X_j^T X_j
  // state
  double *x, *z, *pb0, *pb1, *wc, *K1, *K2, *binv;
  // two-level preconditioner (p entries each; "compact" arrays are indexed by
  // component id, ids < p)
  int* uf;                   // union-find parent of each coefficient
  int* cmap;                 // compact id of each component root
  int* cid;                  // compact id of each coefficient's component, -1 outside any
  int* ncomp;                // number of components of this MM iteration
  double* qcinv;             // 1 / q_c of each coefficient's component (0 outside)
  double *qc, *qci;          // compact: q_c and 1 / q_c
  double *sc0, *sc1;         // compact: component sums of r (alternate CG iterations)
  void* ub0;                 // two accumulators, each kUR replicas of ldn doubles
  void* ub1;                 // (replica r at byte offset 8 * r * ldn; also used as floats)
  double* part;              // [2 slots][kNF][gridDim.x]
  unsigned* bar;
  int* err;
  DevStats* stats;
  long long timeout;
  int inject_stall;          // test hook: block 0 skips the first barrier
};

// Estimated relative error of f(beta) against the exact minimum of Eq. obj:
// the Prop. 1(ii) gap (f - f_eps) / f plus the extrapolated MM tail
// rel * q / (1 - q), q = rel / rel_prev (linear convergence), capped at 0.999.
inline double estimated_error(const DevStats& s) {
  const double f = s.f;
  if (!(f != 0.0) || !std::isfinite(f)) return INFINITY;
  double e = (s.f - s.f_eps) / fabs(f);
  if (e < 0.0) e = 0.0;
  const double rel = s.rel_change, rp = s.rel_prev;
  double tail = rel;
  if (rp > 0.0 && rel > 0.0) {
    double q = rel / rp;
    if (q > 0.999) q = 0.999;
    tail = rel * q / (1.0 - q);
  }
  return e + tail;
}

// Remote stencil neighbours of a block of w consecutive coefficients: the left
// one, the right one, and on a lattice (row length q2 < p) the min(w, q2)
// vertical ones on each side.
__host__ __device__ inline long long halo_entries(long long w, long long q2, long long p) {
  return 2 + (q2 < p ? 2 * (w < q2 ? w : q2) : 0);
}

// Columns of a block's X slab that stay in shared memory for the whole solve:
// as many of its w columns (ldn elements of es bytes each) as fit next to the
// kernel's other shared memory (`base` bytes, rounded up to 16) within dyn_max.
inline int resident_columns(long long w, long long ldn, size_t es, size_t base, int dyn_max) {
  const long long room = (long long)dyn_max - (long long)((base + 15) / 16 * 16);
  if (room <= 0) return 0;
  long long c = room / (ldn * (long long)es);
  return (int)(c < w ? c : w);
}

// shared-memory bytes of mm_solve_kernel (the host uses the same formula)
__host__ __device__ inline size_t solve_smem_bytes(long long ldn, long long wpad, int V, long long nh,
                                                   long long trows = 0) {
  return (size_t)ldn * 8 + (size_t)wpad * 8 + (size_t)kThreads * V * 8 + (size_t)wpad * 8 +
         6 * (size_t)wpad * 8 + 6 * (size_t)wpad * 8 + 6 * (size_t)wpad * 8 +
         ((size_t)kRF * kThreads + 16) * 8 +
         2 * (size_t)nh * 8 + (size_t)nh * 4 +            // halo p values, 1/q_c, component ids
         2 * (size_t)trows * 8 + 8 * 32 * 8 +             // TMEM phase A row partials, phase C partials
         (size_t)wpad * 4 + (size_t)wpad;
}

// ---- X slab columns resident in tensor memory (TMEM).  TMEM is 128 lanes x
// 512 32-bit columns per SM.  Row i of the slab goes to lane i % 128; row
// group g = i / 128 takes cells [g * ct, (g + 1) * ct).  A 32-bit cell holds
// one FP32 element or two 16-bit ones (slab columns 2c and 2c + 1 in its low
// and high halves).  Warp w of the 8 reads lanes 32 (w % 4) .. + 31 (the
// hardware's lane quarters) and cells [(w / 4) ct / 2, (w / 4 + 1) ct / 2) of
// every row group.  Cells per row group (0 = no TMEM): 32 or 64, with at most
// 32 slab columns per half so phase C keeps 32 accumulators per thread.
static_assert(kThreads == 256, "the TMEM layout maps 8 warps onto 4 lane quarters x 2 cell halves");
__host__ __device__ inline int tmem_cells(long long n, int es) {
  if (es != 4 && es != 2) return 0;
  const long long R = (n + 127) / 128;
  long long ct = 512 / R / 32 * 32;
  const long long cap = 64 / (4 / es);
  if (ct > cap) ct = cap;
  return ct >= 32 ? (int)ct : 0;
}

template <typename TX, typename A>
__device__ __forceinline__ void cvt_to(const uint4& raw, A (&o)[XT<TX>::V]) {
  typename XT<TX>::Acc t[XT<TX>::V];
  XT<TX>::cvt(raw, t);
#pragma unroll
  for (int e = 0; e < XT<TX>::V; ++e) o[e] = (A)t[e];
}

// Block sum of F per-thread doubles; threads >= nact must hold zeros.
// rs: kRF*kThreads + 16 doubles.  Every thread returns the totals.
template <int F>
__device__ __forceinline__ void block_reduce(double (&v)[F], double* rs, int nact) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = nact >= kThreads ? kWarps : (nact + 31) / 32;
  if (warp < nw) {
#pragma unroll
    for (int f = 0; f < F; ++f) rs[f * kThreads + tid] = v[f];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int f = 0; f < F; ++f) {
      double s = 0.0;
      for (int k = 0; k < nw; ++k) s += rs[f * kThreads + k * 32 + lane];
      s = warp_sum(s);
      if (lane == 0) rs[kRF * kThreads + f] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int f = 0; f < F; ++f) v[f] = rs[kRF * kThreads + f];
}

// 16 bytes of column jj (block-relative) at element offset `off`: from the
// shared-memory copy for the first ws columns, else streamed from global memory.
__device__ __forceinline__ uint4 lds16(uint32_t a) {
  uint4 r;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(a));
  return r;
}
template <typename TX>
__device__ __forceinline__ uint4 ldx(const TX* __restrict__ Xt, uint32_t xs, int wt, int ws, long long ldn,
                                     long long j0, int jj, long long off) {
  if (jj - wt < ws) return lds16(xs + (uint32_t)(((long long)(jj - wt) * ldn + off) * (long long)sizeof(TX)));
  return ld_stream16(Xt + (j0 + jj) * ldn + off);
}

// raw 32-bit / 16-bit patterns of X elements
template <typename TX> __device__ __forceinline__ uint32_t xbits(const TX* p) {
  if constexpr (sizeof(TX) == 4) return *reinterpret_cast<const uint32_t*>(p);
  else return (uint32_t)*reinterpret_cast<const unsigned short*>(p);
}
// the two elements of a 32-bit cell as A (exact widening)
template <typename TX, typename A>
__device__ __forceinline__ void cell2(uint32_t c, A& lo, A& hi) {
  float a, b;
  if constexpr (std::is_same<TX, __nv_bfloat16>::value) {
    a = __uint_as_float(c << 16);
    b = __uint_as_float(c & 0xffff0000u);
  } else {
    const __half2 h2 = *reinterpret_cast<const __half2*>(&c);
    const float2 f = __half22float2(h2);
    a = f.x; b = f.y;
  }
  lo = (A)a;
  hi = (A)b;
}

// Copy the slab's first wt_l columns into TMEM (rows >= n and columns >= wt_l zero).
template <typename TX>
__device__ __forceinline__ void tmem_fill(uint32_t tmem, const TX* __restrict__ Xt, long long j0, int wt_l,
                                          long long n, long long ldn, int ct) {
  constexpr int cpc = 4 / (int)sizeof(TX);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2, hc = ct / 2;
  const int R = (int)((n + 127) / 128);
  for (int g = 0; g < R; ++g) {
    const long long i = 128LL * g + 32 * q + lane;
    for (int c0 = 0; c0 < hc; c0 += 16) {
      uint32_t r[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int cell = h * hc + c0 + e;
        uint32_t bits = 0;
#pragma unroll
        for (int k = 0; k < cpc; ++k) {
          const int col = cell * cpc + k;
          if (i < n && col < wt_l) bits |= xbits<TX>(Xt + (j0 + col) * ldn + i) << (16 * k);
        }
        r[e] = bits;
      }
      tc::tmem_st16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(g * ct + h * hc + c0), r);
    }
  }
  tc::tmem_wait_st();
}

// TMEM loads wait together: tcgen05.wait::ld covers every load a warp has in
// flight, so phases A and C issue two loads of 16 slab columns per wait.  The
// loads are unconditional (indices clamped to valid cells; surplus results are
// ignored) so their results stay in registers.

// 16 slab columns (16 FP32 cells or 8 cells of 16-bit pairs) of this thread's lane
template <int CPC>
__device__ __forceinline__ void tmem_ld_cols16(uint32_t ta, uint32_t (&r)[16]) {
  if constexpr (CPC == 1) {
    tc::tmem_ld16_raw(ta, r);
  } else {
    tc::tmem_ld8_raw(ta, *reinterpret_cast<uint32_t(*)[8]>(r));
  }
}

// A's partial over 16 slab columns starting at col0 of one loaded chunk
template <typename TX, typename A>
__device__ __forceinline__ A tmem_dot16(const uint32_t (&r)[16], const A* vs, int col0, int wt_l) {
  constexpr int cpc = 4 / (int)sizeof(TX);
  A acc = A(0);
  if constexpr (cpc == 1) {
#pragma unroll
    for (int e = 0; e < 16; ++e)
      if (col0 + e < wt_l) acc = fma((A)__uint_as_float(r[e]), vs[col0 + e], acc);
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      A lo, hi;
      cell2<TX, A>(r[e], lo, hi);
      if (col0 + 2 * e < wt_l) acc = fma(lo, vs[col0 + 2 * e], acc);
      if (col0 + 2 * e + 1 < wt_l) acc = fma(hi, vs[col0 + 2 * e + 1], acc);
    }
  }
  return acc;
}

// Phase A on the TMEM columns: per-row partial sums of X[:, 0:wt_l] v into
// tpa[h * trows + i] (h = the warp's cell half), one wait per row group.
template <typename TX, typename A>
__device__ __forceinline__ void tmem_phase_a(uint32_t tmem, long long n, int ct, int wt_l, const A* vs,
                                             A* tpa, long long trows) {
  constexpr int cpc = 4 / (int)sizeof(TX);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2, hc = ct / 2;
  const int cph = hc * cpc;          // slab columns per half: 16 or 32
  const int R = (int)((n + 127) / 128);
  const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * hc);
  const uint32_t off1 = cph > 16 ? (uint32_t)(16 / cpc) : 0u;   // second chunk (or the first again)
  for (int g = 0; g < R; ++g) {
    uint32_t r0[16], r1[16];
    tmem_ld_cols16<cpc>(tq + (uint32_t)(g * ct), r0);
    tmem_ld_cols16<cpc>(tq + (uint32_t)(g * ct) + off1, r1);
    tc::tmem_wait_ld();
    A acc = tmem_dot16<TX, A>(r0, vs, h * cph, wt_l);
    if (cph > 16) acc += tmem_dot16<TX, A>(r1, vs, h * cph + 16, wt_l);
    tpa[h * trows + 128LL * g + 32 * q + lane] = acc;
  }
}

// Phase C on the TMEM columns: tv[jj] = X[:, jj]^T u for jj < wt_l.  In passes
// of 16 slab columns (two row groups per wait), each thread accumulates its
// rows' products, a shuffle reduce-scatter leaves lanes 2c and 2c + 1 halves of
// the warp's sum for column c of the pass, and the 4 lane quarters add in shared
// memory (tred, 8 x 32 values).
template <typename TX, typename A>
__device__ __forceinline__ void tmem_phase_c(uint32_t tmem, long long n, int ct, int wt_l, const A* us,
                                             double* tred, double* tv) {
  constexpr int cpc = 4 / (int)sizeof(TX);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2, hc = ct / 2;
  const int cph = hc * cpc;   // slab columns per half (<= 32, a multiple of 16)
  const int R = (int)((n + 127) / 128);
  for (int cb = 0; cb < cph; cb += 16) {
    A acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = A(0);
    const uint32_t ta0 = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * hc + cb / cpc);
    auto accum = [&](const uint32_t (&r)[16], int g) {
      const long long i = 128LL * g + 32 * q + lane;
      const A ui = i < n ? us[i] : A(0);
      if constexpr (cpc == 1) {
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = fma((A)__uint_as_float(r[e]), ui, acc[e]);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          A lo, hi;
          cell2<TX, A>(r[e], lo, hi);
          acc[2 * e] = fma(lo, ui, acc[2 * e]);
          acc[2 * e + 1] = fma(hi, ui, acc[2 * e + 1]);
        }
      }
    };
    for (int g0 = 0; g0 < R; g0 += 2) {
      const int g1 = g0 + 1 < R ? g0 + 1 : g0;   // a second row group, or the first again
      uint32_t r0[16], r1[16];
      tmem_ld_cols16<cpc>(ta0 + (uint32_t)(g0 * ct), r0);
      tmem_ld_cols16<cpc>(ta0 + (uint32_t)(g1 * ct), r1);
      tc::tmem_wait_ld();
      accum(r0, g0);
      if (g1 != g0) accum(r1, g1);
    }
    // reduce-scatter of 16 values over the 32 lanes: after the step with offset
    // o a lane keeps the half whose column index has the lane's bit o; column
    // bits 3..0 follow lane bits 4..1, and lanes l, l ^ 1 end with halves
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const int o = 16 >> st, m = 16 >> st;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < m / 2; ++k) {
        const A send = up ? acc[k] : acc[k + m / 2];
        const A keep = up ? acc[k + m / 2] : acc[k];
        acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    if ((lane & 1) == 0) tred[(q * 2 + h) * 32 + cb + (lane >> 1)] = (double)acc[0];
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < wt_l; jj += kThreads) {
    const int hh = jj / cph, c = jj - hh * cph;
    tv[jj] = ((tred[(0 * 2 + hh) * 32 + c] + tred[(1 * 2 + hh) * 32 + c]) +
              (tred[(2 * 2 + hh) * 32 + c] + tred[(3 * 2 + hh) * 32 + c]));
  }
  __syncthreads();
}

// u[0:n] += sum_{j in slab} X[:, j] * v[j - j0]   (v staged in shared memory)
template <typename TX, typename A>
__device__ __forceinline__ void phase_a(const SolveParams& P, const TX* __restrict__ Xt, uint32_t xs,
                                        uint32_t tmem, A* tpa, long long j0, int wl, const A* vs, A* red,
                                        A* u) {
  const int ws = P.ws, wt = P.wt;
  constexpr int V = XT<TX>::V;
  const int tid = threadIdx.x;
  const int nv = (int)(P.ldn / V);
  if (wl <= 0) return;
  const int wt_l = wt < wl ? wt : wl;   // this block's TMEM columns
  const long long trows = (P.n + 127) / 128 * 128;
  if (wt_l > 0) {
    if constexpr (sizeof(TX) == 4 || sizeof(TX) == 2) tmem_phase_a<TX, A>(tmem, P.n, P.tct, wt_l, vs, tpa, trows);
    __syncthreads();
  }
  // per-row TMEM partials (zero without TMEM)
  auto tp = [&](long long i) -> A { return (wt_l > 0 && i < trows) ? tpa[i] + tpa[trows + i] : A(0); };
  if (nv >= kThreads) {
    for (int rv = tid; rv < nv; rv += kThreads) {
      A acc[V];
#pragma unroll
      for (int e = 0; e < V; ++e) acc[e] = tp((long long)rv * V + e);
      const long long off = (long long)rv * V;
      int j = wt_l;
      for (; j + kLA <= wl; j += kLA) {
        uint4 raw[kLA];
#pragma unroll
        for (int k = 0; k < kLA; ++k) raw[k] = ldx<TX>(Xt, xs, wt, ws, P.ldn, j0, j + k, off);
#pragma unroll
        for (int k = 0; k < kLA; ++k) {   // the next group's streamed columns into L2
          const int jn = j + kLA + k;
          if (jn < wl && jn - wt >= ws) prefetch_l2(Xt + (j0 + jn) * P.ldn + off);
        }
#pragma unroll
        for (int k = 0; k < kLA; ++k) {
          A xv[V];
          cvt_to<TX, A>(raw[k], xv);
          const A s = vs[j + k];
#pragma unroll
          for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
        }
      }
      for (; j < wl; ++j) {
        A xv[V];
        cvt_to<TX, A>(ldx<TX>(Xt, xs, wt, ws, P.ldn, j0, j, off), xv);
        const A s = vs[j];
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
      }
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const long long i = (long long)rv * V + e;
        if (i < P.n && acc[e] != A(0)) atomicAdd(u + i, acc[e]);
      }
    }
  } else {
    const int ncg = kThreads / nv;          // column groups, >= 1
    const int rv = tid % nv, cg = tid / nv;
    A acc[V];
#pragma unroll
    for (int e = 0; e < V; ++e) acc[e] = A(0);
    if (cg < ncg) {
      const long long off = (long long)rv * V;
      int j = wt_l + cg;
      for (; j + (kLA - 1) * ncg < wl; j += kLA * ncg) {
        uint4 raw[kLA];
#pragma unroll
        for (int k = 0; k < kLA; ++k) raw[k] = ldx<TX>(Xt, xs, wt, ws, P.ldn, j0, j + k * ncg, off);
#pragma unroll
        for (int k = 0; k < kLA; ++k) {
          A xv[V];
          cvt_to<TX, A>(raw[k], xv);
          const A s = vs[j + k * ncg];
#pragma unroll
          for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
        }
      }
      for (; j < wl; j += ncg) {
        A xv[V];
        cvt_to<TX, A>(ldx<TX>(Xt, xs, wt, ws, P.ldn, j0, j, off), xv);
        const A s = vs[j];
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], s, acc[e]);
      }
#pragma unroll
      for (int e = 0; e < V; ++e) red[cg * nv * V + rv * V + e] = acc[e];
    }
    __syncthreads();
    const int rows = nv * V;
    for (int i = tid; i < rows; i += kThreads) {
      A s = tp(i);
      for (int g = 0; g < ncg; ++g) s += red[g * rows + i];
      if (i < P.n && s != A(0)) atomicAdd(u + i, s);
    }
    __syncthreads();
  }
}

// tv[jj] = X[:, j0+jj]^T u  for jj in [0, wl)   (u staged in shared memory).
// One warp per pair of columns; each lane keeps CPW x UR 16-byte loads in flight.
template <typename TX, typename A>
__device__ __forceinline__ void phase_c(const SolveParams& P, const TX* __restrict__ Xt, uint32_t xs,
                                        uint32_t tmem, double* tred, long long j0, int wl, const A* us,
                                        double* tv) {
  const int ws = P.ws, wt = P.wt;
  const int wt_l = wt < wl ? wt : wl;   // this block's TMEM columns
  if (wt_l > 0) {
    if constexpr (sizeof(TX) == 4 || sizeof(TX) == 2) tmem_phase_c<TX, A>(tmem, P.n, P.tct, wt_l, us, tred, tv);
  }
  constexpr int V = XT<TX>::V;
  constexpr int CPW = 2;  // columns per warp
  constexpr int UR = 4;   // row vectors per lane per round
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = (int)(P.ldn / V);
  for (int base = wt_l + warp * CPW; base < wl; base += kWarps * CPW) {
    A acc[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) acc[c] = A(0);
    for (int rv0 = lane; rv0 < nv; rv0 += 32 * UR) {
      uint4 raw[CPW][UR];
#pragma unroll
      for (int c = 0; c < CPW; ++c)
#pragma unroll
        for (int u = 0; u < UR; ++u) {
          const int rv = rv0 + 32 * u;
          if (base + c < wl && rv < nv)
            raw[c][u] = ldx<TX>(Xt, xs, wt, ws, P.ldn, j0, base + c, (long long)rv * V);
        }
#pragma unroll
      for (int c = 0; c < CPW; ++c)   // the next round's streamed rows into L2
#pragma unroll
        for (int u = 0; u < UR; ++u) {
          const int rvn = rv0 + 32 * (UR + u);
          if (base + c < wl && base + c - wt >= ws && rvn < nv)
            prefetch_l2(Xt + (j0 + base + c) * P.ldn + (long long)rvn * V);
        }
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int rv = rv0 + 32 * u;
        if (rv < nv) {
          A uu[V];
#pragma unroll
          for (int e = 0; e < V; ++e) uu[e] = us[rv * V + e];
#pragma unroll
          for (int c = 0; c < CPW; ++c) {
            if (base + c < wl) {
              A xv[V];
              cvt_to<TX, A>(raw[c][u], xv);
#pragma unroll
              for (int e = 0; e < V; ++e) acc[c] = fma(xv[e], uu[e], acc[c]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const A sum = warp_sum(acc[c]);
      if (lane == 0 && base + c < wl) tv[base + c] = (double)sum;
    }
  }
  __syncthreads();
}

// Precompute the PCR multipliers of the chunk's tridiagonal matrix
// (diagonal `diag`, couplings -lw / -rw between consecutive indices).
__device__ __forceinline__ void setup_tridiag(const SolveParams& P, long long j0, int wl,
                                              const double* diag, const double* lw,
                                              const double* rw, double* sm6) {
  const int tid = threadIdx.x;
  const long long wp = P.wpad;
  double* A0 = sm6;          double* B0 = sm6 + wp;     double* C0 = sm6 + 2 * wp;
  double* A1 = sm6 + 3 * wp; double* B1 = sm6 + 4 * wp; double* C1 = sm6 + 5 * wp;
  for (int jj = tid; jj < wl; jj += kThreads) {
    B0[jj] = diag[jj];
    A0[jj] = jj > 0 ? -lw[jj] : 0.0;
    C0[jj] = jj + 1 < wl ? -rw[jj] : 0.0;
  }
  __syncthreads();
  double *A = A0, *B = B0, *C = C0, *An = A1, *Bn = B1, *Cn = C1;
  for (int l = 0; l < P.levels; ++l) {
    const int s = 1 << l;
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      double k1 = 0.0, k2 = 0.0, bb = B[jj], an = 0.0, cn = 0.0;
      if (jj >= s) {
        k1 = A[jj] / B[jj - s];
        an = -A[jj - s] * k1;
        bb = fma(-C[jj - s], k1, bb);
      }
      if (jj + s < wl) {
        k2 = C[jj] / B[jj + s];
        cn = -C[jj + s] * k2;
        bb = fma(-A[jj + s], k2, bb);
      }
      P.K1[(long long)l * P.p + j] = k1;
      P.K2[(long long)l * P.p + j] = k2;
      An[jj] = an; Bn[jj] = bb; Cn[jj] = cn;
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

// z = M^-1 r for the block's own coefficients: r from shared memory, z to
// shared memory and to global memory (neighbouring blocks read it as halo).
// Jacobi: r / diag(Q).  Tridiagonal: parallel cyclic reduction with the
// multipliers precomputed once per MM iteration (K1, K2, binv).
__device__ __forceinline__ void apply_precond(const SolveParams& P, bool tri, long long j0, int wl,
                                              const double* sidg, const double* rsm,
                                              double* zsm, double* w0, double* w1) {
  const int tid = threadIdx.x;
  if (!tri) {
    for (int jj = tid; jj < wl; jj += kThreads) {
      const double z = rsm[jj] * sidg[jj];
      zsm[jj] = z;
      P.z[j0 + jj] = z;
    }
    __syncthreads();
    return;
  }
  for (int jj = tid; jj < wl; jj += kThreads) w0[jj] = rsm[jj];
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
  for (int jj = tid; jj < wl; jj += kThreads) {
    const double z = cur[jj] * P.binv[j0 + jj];
    zsm[jj] = z;
    P.z[j0 + jj] = z;
  }
  __syncthreads();
}

// Sum the kUR replicas of an n-vector accumulator (ldn entries each, padding
// zero; replica r at byte offset 8 * r * ldn) into shared memory with 16-byte
// coherent loads, in a fixed replica order; returns this thread's partial sum
// of squares of the first n entries (FP64), or of (y - u)^2 when `resid`.
template <typename A>
__device__ __forceinline__ double stage_u(const A* __restrict__ u, A* us, long long n, long long ldn,
                                          const double* y, bool resid) {
  constexpr int VA = 16 / sizeof(A);
  const int nvec = (int)(ldn / VA);
  const long long rstride = ldn * 8 / (long long)sizeof(A);   // elements between replicas
  double acc = 0.0;
  for (int v = threadIdx.x; v < nvec; v += kThreads) {
    A t[VA];
#pragma unroll
    for (int e = 0; e < VA; ++e) t[e] = A(0);
#pragma unroll
    for (int r = 0; r < kUR; ++r) {
      if constexpr (VA == 4) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(u + r * rstride) + v);
        t[0] += (A)q.x; t[1] += (A)q.y; t[2] += (A)q.z; t[3] += (A)q.w;
      } else {
        const double2 q = __ldcg(reinterpret_cast<const double2*>(u + r * rstride) + v);
        t[0] += (A)q.x; t[1] += (A)q.y;
      }
    }
#pragma unroll
    for (int e = 0; e < VA; ++e) {
      const long long i = (long long)v * VA + e;
      if (i < n) {
        us[i] = t[e];
        const double d = resid ? y[i] - (double)t[e] : (double)t[e];
        acc = fma(d, d, acc);
      } else {
        us[i] = A(0);
      }
    }
  }
  return acc;
}

// ---- union-find over the strong edges (PC_TWOLEVEL): lock-free hooking of
// the larger root under the smaller one by CAS, with path halving (the
// ECL-CC scheme, Jaiganesh and Burtscher 2018).  Parent pointers never
// increase (par[x] <= x), so every walk ends within x + 1 steps.
__device__ __forceinline__ int vld(const int* a) { return *reinterpret_cast<const volatile int*>(a); }
__device__ __forceinline__ void vst(int* a, int v) { *reinterpret_cast<volatile int*>(a) = v; }

__device__ __forceinline__ int uf_root(int* par, int x, bool halve) {
  int cur = x;
  for (int it = 0; it <= x; ++it) {
    const int pc = vld(par + cur);
    if (pc == cur) break;
    const int gp = vld(par + pc);
    if (halve && gp != pc) vst(par + cur, gp);
    cur = gp;
  }
  return cur;
}

// merge the components of a and b; each failed CAS lowers the larger root,
// so the loop ends within `bound` rounds
__device__ __forceinline__ void uf_union(int* par, int a, int b, long long bound) {
  a = uf_root(par, a, true);
  b = uf_root(par, b, true);
  for (long long it = 0; a != b && it <= bound; ++it) {
    if (a < b) { const int t = a; a = b; b = t; }
    const int old = atomicCAS(par + a, a, b);
    if (old == a) return;
    a = uf_root(par, old, true);
    b = uf_root(par, b, true);
  }
}

// acc[key] += v over the lanes with key >= 0, one atomic per distinct key of
// the warp.  All 32 lanes must call it.
__device__ __forceinline__ void warp_add_by_key(double* acc, int key, double v) {
  const int lane = threadIdx.x & 31;
  unsigned pend = __ballot_sync(0xffffffffu, key >= 0);
  while (pend) {
    const int l = __ffs(pend) - 1;
    const int k = __shfl_sync(0xffffffffu, key, l);
    const bool mine = key == k;
    const double s = warp_sum(mine ? v : 0.0);
    if (lane == l) atomicAdd(acc + k, s);
    pend &= ~__ballot_sync(0xffffffffu, mine);
  }
}

__device__ __forceinline__ double edge_w(double xj, double xk, double eps) {
  return 1.0 / (fabs(xj - xk) + eps);
}

template <typename TX, int GK, bool CH>
__device__ __forceinline__ void mm_solve_body(const SolveParams& P, uint32_t tmem) {
  using Acc = typename XT<TX>::Acc;
  constexpr int V = XT<TX>::V;
  // X = I: n = p, X^T y = y, X^T X = I; the X products become the vector itself
  constexpr bool IDX = std::is_same<TX, IdX>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tid = threadIdx.x;
  const int G = gridDim.x, b = blockIdx.x;
  const long long p = P.p, n = P.n, q2 = P.q2;
  const long long j0 = (long long)b * P.w;
  const long long j1 = j0 + P.w < p ? j0 + P.w : p;
  const int wl = j1 > j0 ? (int)(j1 - j0) : 0;
  const int ncol = wl < kThreads ? wl : kThreads;          // threads holding column data
  const long long wp = P.wpad;

  // shared memory (solve_smem_bytes)
  double* usd = reinterpret_cast<double*>(smraw);           // ldn: u staged (double or Acc)
  double* vsd = usd + P.ldn;                                // wpad: vector slab (double or Acc)
  double* redd = vsd + wp;                                  // kThreads*V: phase A partials
  double* tv = redd + (long long)kThreads * V;              // wpad: X^T u per column
  double* pw = tv + wp;                                     // 6*wpad: PCR work
  double* cst = pw + 6 * wp;                                // 6*wpad: per-column constants
  double* own = cst + 6 * wp;                               // 6*wpad: own CG vectors
  double* rs = own + 6 * wp;                                // kRF*kThreads + 16
  const long long nh = halo_entries(wp, q2, p);
  double* hv = rs + kRF * kThreads + 16;                    // nh: p at the remote neighbours
  double* hq = hv + nh;                                     // nh: their 1/q_c
  const long long trows = P.tct > 0 ? (n + 127) / 128 * 128 : 0;
  double* tpa = hq + nh;                                    // 2*trows: TMEM phase A row partials
  double* tred = tpa + 2 * trows;                           // 8*32: TMEM phase C partials
  int* cid_s = reinterpret_cast<int*>(tred + 8 * 32);                             // wpad
  int* hc = cid_s + wp;                                                           // nh
  unsigned char* nb = reinterpret_cast<unsigned char*>(hc + nh);                  // wpad
  // ws leading columns of the slab, resident for the whole solve (16-byte aligned)
  const size_t xs_off = (solve_smem_bytes(P.ldn, wp, V, nh, trows) + 15) / 16 * 16;
  const uint32_t xs_sh = (uint32_t)__cvta_generic_to_shared(smraw) + (uint32_t)xs_off;
  // The component sums of r of the last CG iteration, copied to shared memory
  // after its barrier 2 when nc <= kThreads * V; they share the phase A partials'
  // space, which holds nothing between phase A and the next iteration's.
  double* scs = redd;
  const int sc_cap = kThreads * V;
  // remote halo: slot 0 the left neighbour of the first owned coefficient, 1 the
  // right neighbour of the last, then hn up and hn down neighbours (lattice)
  const int hn = (q2 < p) ? (int)(wl < q2 ? wl : q2) : 0;
  const int hd0 = (wl > q2) ? (int)(wl - q2) : 0;           // first jj whose down neighbour is remote
  double* s_la = cst;            // lam1 a_j
  double* s_wl = cst + wp;       // lam2 w(j-1, j) etc.
  double* s_wr = cst + 2 * wp;
  double* s_wu = cst + 3 * wp;
  double* s_wd = cst + 4 * wp;
  double* s_idg = cst + 5 * wp;  // 1 / diag(Q)
  double* xs = own;              // x (also written to global for the halo of the reweight)
  double* rsm = own + wp;        // r
  double* zs = own + 2 * wp;     // z (also global: halo of p)
  double* ps = own + 3 * wp;     // p (also global, double-buffered)
  double* qs = own + 4 * wp;     // S p  (S x at the CG start)
  double* qi_s = own + 5 * wp;   // 1 / q_c of the coefficient's component (PC_TWOLEVEL)
  double* sc = rs + kRF * kThreads + 8;   // scalar broadcast slots
  Acc* us = reinterpret_cast<Acc*>(usd);
  Acc* vs = reinterpret_cast<Acc*>(vsd);
  Acc* red = reinterpret_cast<Acc*>(redd);

  const TX* Xt = reinterpret_cast<const TX*>(P.Xt);
  const unsigned long long t_kernel0 = (b == 0 && tid == 0) ? global_ns() : 0ull;
  GridBarrier gb{P.bar, P.err, 0u, P.timeout};
  SplitBarrier sb{P.cbar, P.err, {0u, 0u}, P.timeout};
  int slot = 0;
  const long long zchunk = (n + G - 1) / G;
  const long long zs0 = (long long)b * zchunk;
  const long long ze0 = zs0 + zchunk < n ? zs0 + zchunk : n;

  // grid-wide sum of F fields: every block contributes v and receives totals
  auto grid_sum = [&](auto& v) -> bool {
    constexpr int F = sizeof(v) / sizeof(double);
    if (tid == 0) {
#pragma unroll
      for (int f = 0; f < F; ++f) P.part[((long long)slot * kNF + f) * G + b] = v[f];
    }
    if (!gb.sync()) return false;
#pragma unroll
    for (int f = 0; f < F; ++f)
      v[f] = tid < G ? ldcg(&P.part[((long long)slot * kNF + f) * G + tid]) : 0.0;
    block_reduce<F>(v, rs, G);
    slot ^= 1;
    return true;
  };
  auto zero_u = [&](void* buf) {   // this block's chunk of every replica
    double* u = reinterpret_cast<double*>(buf);
    for (int r = 0; r < kUR; ++r)
      for (long long i = zs0 + tid; i < ze0; i += kThreads) u[(long long)r * P.ldn + i] = 0.0;
  };
  const int rep = b % kUR;   // this block's accumulator replica
  const bool two = P.precond == PC_TWOLEVEL;
  // local part of M: the chunk-tridiagonal solve (TRIDIAG, PAPER, and TWOLEVEL
  // on a chain), else the diagonal
  const bool tri = GK == GK_STENCIL &&
                   (P.precond == PC_TRIDIAG || P.precond == PC_PAPER || (two && P.q2 >= P.p));
  const int lane = tid & 31, warp = tid >> 5;

  // ---- the slab's first wt columns into TMEM, the next ws into shared memory
  if constexpr (sizeof(TX) == 4 || sizeof(TX) == 2) {
    if (P.tct > 0) tmem_fill<TX>(tmem, Xt, j0, P.wt < wl ? P.wt : wl, n, P.ldn, P.tct);
  }
  if constexpr (!IDX) {
    const int left = wl - P.wt;               // the last block may own fewer columns
    const int wsl = P.ws < left ? P.ws : (left > 0 ? left : 0);
    const long long nvec = (long long)wsl * P.ldn * (long long)sizeof(TX) / 16;
    const uint4* src = reinterpret_cast<const uint4*>(Xt + (j0 + P.wt) * P.ldn);
    uint4* dst = reinterpret_cast<uint4*>(smraw + xs_off);
    for (long long v = tid; v < nvec; v += kThreads) dst[v] = __ldg(src + v);
  }
  // ---- initialisation (Algorithm 1): beta_j = X_j^T y / X_j^T X_j
  for (int jj = tid; jj < wl; jj += kThreads) {
    const long long j = j0 + jj;
    double v;
    if (P.beta_init) v = P.beta_init[j];
    else v = P.d[j] != 0.0 ? P.c[j] / P.d[j] : 0.0;
    P.x[j] = v;
    unsigned char fl = 0;
    if (GK == GK_STENCIL) {
      const long long col = j % q2;
      if (col != 0) fl |= NB_L;
      if (col != q2 - 1 && j + 1 < p) fl |= NB_R;
      if (j >= q2) fl |= NB_U;
      if (j + q2 < p) fl |= NB_D;
    }
    nb[jj] = fl;
  }
  if (P.inject_stall && b == 0) return;   // the others' bounded waits must expire
  if (!gb.sync()) return;

  int ucur = 0, pcur = 0, mm = 0, cg_total = 0, status = ST_OK, nref_total = 0;
  double f = 0.0, f_prev = 0.0, rel = 0.0, rel_prev = 0.0, relres = 0.0, rss_last = 0.0;
  // true when accumulator buffer `ucur` already holds X x for the current x in
  // FP64 (left by the last refinement pass), so the next MM iteration skips it
  bool u0_ready = false;

  while (true) {
    void* U0 = ucur ? P.ub1 : P.ub0;
    void* U1 = ucur ? P.ub0 : P.ub1;
    // ---------------- reweight (Eq. lin-sys), S x, penalties of f
    double pen[2] = {0.0, 0.0};   // sum|x_j|, sum_E|x_j - x_k|
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      const double xj = ldcg(P.x + j);
      const double aj = 1.0 / (fabs(xj) + P.eps);
      double deg = 0.0, lap = 0.0;
      if (GK == GK_STENCIL) {
        const unsigned char fl = nb[jj];
        double wl_ = 0.0, wr_ = 0.0, wu_ = 0.0, wd_ = 0.0;
        const double xl = (fl & NB_L) ? ldcg(P.x + j - 1) : 0.0;
        const double xr = (fl & NB_R) ? ldcg(P.x + j + 1) : 0.0;
        const double xu = (fl & NB_U) ? ldcg(P.x + j - q2) : 0.0;
        const double xd = (fl & NB_D) ? ldcg(P.x + j + q2) : 0.0;
        if (fl & NB_L) { wl_ = edge_w(xl, xj, P.eps); lap = fma(wl_, xj - xl, lap); }
        if (fl & NB_R) { wr_ = edge_w(xj, xr, P.eps); lap = fma(wr_, xj - xr, lap); pen[1] += fabs(xj - xr); }
        if (fl & NB_U) { wu_ = edge_w(xu, xj, P.eps); lap = fma(wu_, xj - xu, lap); }
        if (fl & NB_D) { wd_ = edge_w(xj, xd, P.eps); lap = fma(wd_, xj - xd, lap); pen[1] += fabs(xj - xd); }
        deg = (wl_ + wr_) + (wu_ + wd_);
        s_wl[jj] = P.lam2 * wl_; s_wr[jj] = P.lam2 * wr_;
        s_wu[jj] = P.lam2 * wu_; s_wd[jj] = P.lam2 * wd_;
        if (two) {   // strong edges: the same test, with the same operands, at both ends
          const double dlj = fma(P.lam1, aj, P.d[j]);
          auto strong = [&](double lw, long long kk, double xk) {
            return lw >= kStrong * fmin(dlj, fma(P.lam1, 1.0 / (fabs(xk) + P.eps), P.d[kk]));
          };
          unsigned char sb = fl & 15;
          if ((fl & NB_L) && strong(s_wl[jj], j - 1, xl)) sb |= NB_SL;
          if ((fl & NB_R) && strong(s_wr[jj], j + 1, xr)) sb |= NB_SR;
          if ((fl & NB_U) && strong(s_wu[jj], j - q2, xu)) sb |= NB_SU;
          if ((fl & NB_D) && strong(s_wd[jj], j + q2, xd)) sb |= NB_SD;
          nb[jj] = sb;
          P.uf[j] = (int)j;
        }
      } else {
        const double dlj = fma(P.lam1, aj, P.d[j]);
        bool any_strong = false;
        for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e) {
          const long long k = P.col[e];
          const double xk = ldcg(P.x + k);
          const double we = k > j ? edge_w(xj, xk, P.eps) : edge_w(xk, xj, P.eps);
          P.wc[e] = P.lam2 * we;
          deg += we;
          lap = fma(we, xj - xk, lap);
          if (k > j) pen[1] += fabs(xj - xk);
          if (two && P.lam2 * we >= kStrong * fmin(dlj, fma(P.lam1, 1.0 / (fabs(xk) + P.eps), P.d[k])))
            any_strong = true;
        }
        if (two) {
          nb[jj] = any_strong ? NB_SR : 0;
          P.uf[j] = (int)j;
        }
      }
      pen[0] += fabs(xj);
      const double la = P.lam1 * aj;
      s_la[jj] = la;
      const double dq = fma(P.lam2, deg, la + P.d[j]);
      s_idg[jj] = 1.0 / dq;
      qs[jj] = fma(la, xj, P.lam2 * lap);      // S x
      tv[jj] = (P.precond == PC_PAPER) ? dq - P.d[j] : dq;   // tridiagonal diagonal
      vsd[jj] = xj;
      xs[jj] = xj;
    }
    __syncthreads();
    if (tri) setup_tridiag(P, j0, wl, tv, s_wl, s_wr, pw);
    // ---------------- u0 = X x in FP64 (refinement pass)
    double pr3[3] = {pen[0], pen[1], 0.0};   // penalties, and ||y - x||^2 when X = I
    if constexpr (!IDX) {
      zero_u(U1);
      if (!u0_ready)
        phase_a<TX, double>(P, Xt, xs_sh, tmem, tpa, j0, wl, vsd, redd, reinterpret_cast<double*>(U0) + (long long)rep * P.ldn);
    } else {
      for (int jj = tid; jj < wl; jj += kThreads) {
        const double d = P.y[j0 + jj] - xs[jj];
        pr3[2] = fma(d, d, pr3[2]);
      }
    }
    u0_ready = false;
    block_reduce<3>(pr3, rs, ncol);
    if (!grid_sum(pr3)) return;
    pen[0] = pr3[0];
    pen[1] = pr3[1];
    // ---------------- f(beta(r)) (Eq. obj) and the outer stop test
    if constexpr (!IDX) {
      double rv[1] = {stage_u<double>(reinterpret_cast<const double*>(U0), usd, n, P.ldn, P.y, true)};
      block_reduce<1>(rv, rs, kThreads);
      rss_last = rv[0];
    } else {
      rss_last = pr3[2];
    }
    f = 0.5 * rss_last + P.lam1 * pen[0] + P.lam2 * pen[1];
    if (!isfinite(f)) { status = ST_NONFINITE; break; }
    if (mm > 0) {
      rel_prev = rel;
      rel = fabs(f - f_prev) / fabs(f_prev);
      if (rel <= P.tol) break;
    }
    if (mm >= P.max_mm) { status = ST_NOTCONV; break; }
    // inner tolerance of this MM iteration
    const double tol_in = fmax(P.tol_cg, P.tol_cg_rel * (mm > 0 ? rel : 1.0));
    // ---------------- r0 = c - Q x0 (FP64), z0 = M^-1 r0, p1 = z0 (Algorithm 2)
    if constexpr (!IDX) phase_c<TX, double>(P, Xt, xs_sh, tmem, tred, j0, wl, usd, tv);
    else for (int jj = tid; jj < wl; jj += kThreads) tv[jj] = xs[jj];
    for (int jj = tid; jj < wl; jj += kThreads) rsm[jj] = (P.c[j0 + jj] - tv[jj]) - qs[jj];
    __syncthreads();
    int nc = 0;   // coarse components of this MM iteration (PC_TWOLEVEL)
    if (two) {
      // the compact arrays are free: their last readers finished before the
      // grid barrier of the refinement pass.  Block ranges jointly cover [0, p).
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        P.qc[j] = 0.0;
        P.sc0[j] = 0.0;
        P.sc1[j] = 0.0;
      }
      if (b == 0 && tid == 0) vst(P.ncomp, 0);
      // union over the strong edges, each from its lower end
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        const unsigned char fl = nb[jj];
        if (GK == GK_STENCIL) {
          if (fl & NB_SR) uf_union(P.uf, (int)j, (int)(j + 1), p);
          if (fl & NB_SD) uf_union(P.uf, (int)j, (int)(j + q2), p);
        } else if (fl & NB_SR) {   // the reweight's strong test, recomputed per edge
          const double dlj = fma(P.lam1, 1.0 / (fabs(xs[jj]) + P.eps), P.d[j]);
          for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e) {
            const long long kk = P.col[e];
            if (kk < j) continue;
            const double dlk = fma(P.lam1, 1.0 / (fabs(ldcg(P.x + kk)) + P.eps), P.d[kk]);
            if (P.wc[e] >= kStrong * fmin(dlj, dlk)) uf_union(P.uf, (int)j, (int)kk, p);
          }
        }
      }
      if (!gb.sync()) return;
      // roots are final: point every coefficient at its root; each root of a
      // component of size >= 2 (exactly the coefficients with a strong edge)
      // takes a compact id
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        const int r = uf_root(P.uf, (int)j, false);
        vst(P.uf + j, r);
        if (r == (int)j && (nb[jj] & NB_STRONG)) P.cmap[j] = atomicAdd(P.ncomp, 1);
      }
      if (!gb.sync()) return;
      nc = vld(P.ncomp);
      // labels, q_c and the component sums of r0
      for (int base = warp * 32; base < wl; base += kThreads) {   // warp-uniform trip count
        const int jj = base + lane;
        int key = -1;
        double qv = 0.0, rv = 0.0;
        if (jj < wl) {
          const long long j = j0 + jj;
          const unsigned char fl = nb[jj];
          if (fl & NB_STRONG) {
            const int r = vld(P.uf + j);
            const int c = (r >= 0 && r < p) ? P.cmap[r] : -1;
            if (c >= 0 && c < nc) {
              key = c;
              double qv_ = s_la[jj] + P.d[j];   // plus lam2 w of the edges leaving the component
              if (GK == GK_STENCIL) {
                if ((fl & NB_L) && vld(P.uf + j - 1) != r) qv_ += s_wl[jj];
                if ((fl & NB_R) && vld(P.uf + j + 1) != r) qv_ += s_wr[jj];
                if ((fl & NB_U) && vld(P.uf + j - q2) != r) qv_ += s_wu[jj];
                if ((fl & NB_D) && vld(P.uf + j + q2) != r) qv_ += s_wd[jj];
              } else {
                for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e)
                  if (vld(P.uf + P.col[e]) != r) qv_ += P.wc[e];
              }
              qv = qv_;
              rv = rsm[jj];
            }
          }
          cid_s[jj] = key;
          P.cid[j] = key;
        }
        warp_add_by_key(P.qc, key, qv);
        warp_add_by_key(P.sc0, key, rv);
      }
      if (!gb.sync()) return;
      for (int jj = tid; jj < wl; jj += kThreads) {
        const int c = cid_s[jj];
        const double qi = c >= 0 ? 1.0 / ldcg(P.qc + c) : 0.0;
        qi_s[jj] = qi;
        P.qcinv[j0 + jj] = qi;
      }
      for (long long c = j0 + tid; c < j1 && c < nc; c += kThreads) P.qci[c] = 1.0 / ldcg(P.qc + c);
      __syncthreads();
    }
    // The inner solve.  Each pass runs PCG from the residual in rsm (whose
    // component sums are in the array picked by kpar) until the recursive
    // residual meets tol_cg; with max_refine > 0 the true residual
    // c - Q x is then recomputed in FP64 and, while it is still above
    // tol_cg, PCG restarts from it (mixed-precision iterative refinement of
    // one surrogate system).
    int kpar = 0;        // CG iteration k accumulates component sums into sc[(k + kpar + 1) & 1]
    int nref_mm = 0, cg_mm = 0;
    while (true) {
      double* Sr = (kpar & 1) ? P.sc1 : P.sc0;   // component sums of the start residual
      apply_precond(P, tri, j0, wl, s_idg, rsm, zs, pw, pw + wp);
      if (two) {   // z0 = D^-1 r0 + coarse part
        for (int jj = tid; jj < wl; jj += kThreads) {
          const int c = cid_s[jj];
          if (c >= 0) zs[jj] = fma(ldcg(Sr + c), qi_s[jj], zs[jj]);
        }
        __syncthreads();
      }
      double rz2[2] = {0.0, 0.0};
      {
        double* pg = pcur ? P.pb1 : P.pb0;
        for (int jj = tid; jj < wl; jj += kThreads) {
          const double rj = rsm[jj], zj = zs[jj];
          ps[jj] = zj;
          pg[j0 + jj] = zj;
          rz2[0] = fma(rj, zj, rz2[0]);
          rz2[1] = fma(rj, rj, rz2[1]);
        }
      }
      block_reduce<2>(rz2, rs, ncol);
      if (!grid_sum(rz2)) return;
      double rz = rz2[0], rr = rz2[1], gamma = 0.0;
      // the adaptive tolerance never lets an inner solve stop before it has halved
      // its start residual (an inexact-Newton safeguard), so every MM iteration
      // makes progress
      // (kept in the shared scalar slot sc[5], read by the deciding thread)
      if (tid == 0) sc[5] = P.tol_cg_rel > 0.0 ? fmax(P.tol_cg, fmin(tol_in, 0.5 * sqrt(rr) / P.cnorm)) : P.tol_cg;
      ucur ^= 1;
      // ---------------- CG iterations (inner products and scalars in FP64)
      int k = 0;
      while (true) {
        if (tid == 0) {
          const double rel_r = sqrt(rr) / P.cnorm;
          sc[0] = rel_r;
          sc[1] = (k >= P.max_cg || (k >= P.min_cg && rel_r <= sc[5])) ? 1.0 : 0.0;
        }
        __syncthreads();
        relres = sc[0];
        if (sc[1] != 0.0) break;
        Acc* Ucur = reinterpret_cast<Acc*>(ucur ? P.ub1 : P.ub0);
        void* Unext = ucur ? P.ub0 : P.ub1;
        const double* pc = pcur ? P.pb1 : P.pb0;
        const double* po = pcur ? P.pb0 : P.pb1;
        // component sums of r: this iteration's accumulator and the previous one's
        double* Scur = ((k + kpar) & 1) ? P.sc0 : P.sc1;
        double* Sold = ((k + kpar) & 1) ? P.sc1 : P.sc0;
        // p at a neighbour: own values from shared memory; another block's value is
        // z + gamma p_old (bit-identical to its owner's update), or p itself at k = 0
        auto pval = [&](long long kk) -> double {
          if (kk >= j0 && kk < j1) return ps[kk - j0];
          if (k == 0) return ldcg(pc + kk);
          double zk = ldcg(P.z + kk);
          if (two) {
            const int c = __ldcg(P.cid + kk);
            if (c >= 0) zk = fma(ldcg(Sold + c), ldcg(P.qcinv + kk), zk);
          }
          return fma(gamma, ldcg(po + kk), zk);
        };
        // component sums of the previous iteration: the shared-memory copy made
        // after its barrier 2 when they fit, else global memory
        const bool sc_smem = nc <= sc_cap;
        if (GK == GK_STENCIL) {
          // p at the block's remote neighbours, every load of the block in flight at
          // once (z + coarse part + gamma p_old as in pval, or p itself at k = 0);
          // 1/q_c and component ids of remote neighbours are fetched at k = 0 and
          // kept for the rest of the MM iteration
          for (int e = tid; e < 2 + 2 * hn; e += kThreads) {
            long long kk;
            unsigned char bit;
            if (e == 0) { kk = j0 - 1; bit = NB_L; }
            else if (e == 1) { kk = j1; bit = NB_R; }
            else if (e < 2 + hn) { kk = j0 + (e - 2) - q2; bit = NB_U; }
            else { kk = j0 + hd0 + (e - 2 - hn) + q2; bit = NB_D; }
            const int jj = e == 0 ? 0 : e == 1 ? wl - 1 : e < 2 + hn ? e - 2 : hd0 + (e - 2 - hn);
            if (wl == 0 || !(nb[jj] & bit)) continue;
            double v;
            if (k == 0) {
              v = ldcg(pc + kk);
              if (two) { hc[e] = __ldcg(P.cid + kk); hq[e] = ldcg(P.qcinv + kk); }
            } else {
              double zk = ldcg(P.z + kk);
              const double pk = ldcg(po + kk);
              if (two) {
                const int c = hc[e];
                if (c >= 0) zk = fma(sc_smem ? scs[c] : ldcg(Sold + c), hq[e], zk);
              }
              v = fma(gamma, pk, zk);
            }
            hv[e] = v;
          }
          __syncthreads();
        }
        double sv[2] = {0.0, 0.0};   // p^T S p, and ||p||^2 when X = I
        for (int jj = tid; jj < wl; jj += kThreads) {
          const long long j = j0 + jj;
          const double pj = ps[jj];
          double lap = 0.0;
          if (GK == GK_STENCIL) {
            const unsigned char fl = nb[jj];
            const double pl = (fl & NB_L) ? (jj == 0 ? hv[0] : ps[jj - 1]) : pj;
            const double pr = (fl & NB_R) ? (jj == wl - 1 ? hv[1] : ps[jj + 1]) : pj;
            const double pu = (fl & NB_U) ? (jj < q2 ? hv[2 + jj] : ps[jj - q2]) : pj;
            const double pd = (fl & NB_D) ? (jj >= hd0 ? hv[2 + hn + jj - hd0] : ps[jj + q2]) : pj;
            lap = fma(s_wl[jj], pj - pl, lap);
            lap = fma(s_wr[jj], pj - pr, lap);
            lap = fma(s_wu[jj], pj - pu, lap);
            lap = fma(s_wd[jj], pj - pd, lap);
          } else {
            for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e)
              lap = fma(P.wc[e], pj - pval(P.col[e]), lap);
          }
          const double spj = fma(s_la[jj], pj, lap);
          qs[jj] = spj;
          sv[0] = fma(pj, spj, sv[0]);
          if constexpr (IDX) sv[1] = fma(pj, pj, sv[1]);   // ||X p||^2 = ||p||^2
          vs[jj] = (Acc)pj;
        }
        double uu[1] = {0.0};
        bool tv_done = false;   // the chunked Q-apply leaves X^T u in tv
        if constexpr (!IDX) {
          if constexpr (CH) {
            // One pass over X: for row chunk s, phase A of chunk s streams from
            // HBM and adds into u; after the split barrier of chunk s - 1 (whose
            // wait overlaps the streaming), phase C of chunk s - 1 re-reads that
            // chunk from L2.  Each thread owns row vector rv of every chunk and the
            // slab columns cg, cg + kCCG, ....  p^T S p rides on the barrier of
            // chunk 0.
            constexpr int Rc = kCRV * V;
            const int rv = tid % kCRV, cg = tid / kCRV;
            const int ncols = wl > cg ? (wl - cg + kCCG - 1) / kCCG : 0;
            const int nch = (int)((n + Rc - 1) / Rc);
            Acc* red_c = red;
            zero_u(Unext);
            if (tid == 0) P.part[((long long)slot * kNF) * G + b] = 0.0;
            {
              double sv1[1] = {sv[0]};
              block_reduce<1>(sv1, rs, ncol);
              if (tid == 0) P.part[((long long)slot * kNF) * G + b] = sv1[0];
            }
            // X^T u accumulates in tv: after each chunk, a column's partials are
            // summed over the kCRV row-vector lanes by shuffles (the two column
            // groups of a warp loop to the larger count; lanes past their own
            // count add zeros) and lane rv == 0 adds the sum to tv.
            const int ncols_w = wl > (cg & ~1) ? (wl - (cg & ~1) + kCCG - 1) / kCCG : 0;
            if (rv == 0)
              for (int c = 0; c < ncols; ++c) tv[cg + c * kCCG] = 0.0;
            double uu_loc = 0.0;
            auto colptr = [&](int c, long long off) { return Xt + (j0 + cg + (long long)c * kCCG) * P.ldn + off; };
            bool ok = true;
            for (int st = 0; st <= nch && ok; ++st) {
              if (st < nch) {   // phase A of chunk st
                const long long off = (long long)(st * kCRV + rv) * V;
                const bool rowok = off < P.ldn;
                Acc acc[V];
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = Acc(0);
#pragma unroll 1
                for (int c0 = 0; c0 < ncols; c0 += kLC) {
                  uint4 raw[kLC];
#pragma unroll
                  for (int k = 0; k < kLC; ++k)
                    if (c0 + k < ncols && rowok) raw[k] = ld_stream16(colptr(c0 + k, off));
#pragma unroll
                  for (int k = 0; k < kLC; ++k) {
                    if (c0 + k < ncols && rowok) {
                      Acc xv[V];
                      cvt_to<TX, Acc>(raw[k], xv);
                      const Acc sp = vs[cg + (c0 + k) * kCCG];
#pragma unroll
                      for (int e = 0; e < V; ++e) acc[e] = fma(xv[e], sp, acc[e]);
                    }
                  }
                }
#pragma unroll
                for (int e = 0; e < V; ++e) red_c[cg * Rc + rv * V + e] = acc[e];
                __syncthreads();
                for (int i = tid; i < Rc; i += kThreads) {
                  Acc sum = Acc(0);
                  for (int g = 0; g < kCCG; ++g) sum += red_c[g * Rc + i];
                  const long long row = (long long)st * Rc + i;
                  if (row < n && sum != Acc(0)) atomicAdd(Ucur + row, sum);
                }
                sb.arrive(st);
              }
              if (st > 0) {     // phase C of chunk st - 1
                if (!sb.wait(st - 1)) { ok = false; break; }
                if (st == 1) {  // p^T S p from the partials published before barrier 0
                  double v1[1] = {tid < G ? ldcg(&P.part[((long long)slot * kNF) * G + tid]) : 0.0};
                  block_reduce<1>(v1, rs, G);
                  sv[0] = v1[0];
                }
                const long long off = (long long)((st - 1) * kCRV + rv) * V;
                const bool rowok = off < P.ldn;
                Acc ul[V];
#pragma unroll
                for (int e = 0; e < V; ++e) {
                  const long long row = off + e;
                  ul[e] = (rowok && row < n) ? ldcg(Ucur + row) : Acc(0);
                  if (cg == 0) uu_loc = fma((double)ul[e], (double)ul[e], uu_loc);
                }
#pragma unroll 1
                for (int c0 = 0; c0 < ncols_w; c0 += kLCC) {
                  uint4 raw[kLCC];
#pragma unroll
                  for (int k = 0; k < kLCC; ++k)
                    if (c0 + k < ncols && rowok) raw[k] = ld_stream16(colptr(c0 + k, off));
                  Acc d[kLCC];
#pragma unroll
                  for (int k = 0; k < kLCC; ++k) {
                    d[k] = Acc(0);
                    if (c0 + k < ncols && rowok) {
                      Acc xv[V];
                      cvt_to<TX, Acc>(raw[k], xv);
#pragma unroll
                      for (int e = 0; e < V; ++e) d[k] = fma(xv[e], ul[e], d[k]);
                    }
                  }
                  // reduce-scatter over the kCRV lanes: each halving step keeps the
                  // upper or lower half of the columns, then the remaining lanes of
                  // a group all-reduce; lane rv ends with column col
                  int col = 0;
                  int m = kLCC;
#pragma unroll
                  for (int o = kCRV / 2; o >= 1; o >>= 1) {
                    if (m > 1) {
                      const bool hi = (rv & o) != 0;
#pragma unroll
                      for (int i = 0; i < kLCC / 2; ++i) {
                        if (i < m / 2) {
                          const Acc send = hi ? d[i] : d[i + m / 2];
                          const Acc keep = hi ? d[i + m / 2] : d[i];
                          d[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                        }
                      }
                      if (hi) col += m / 2;
                      m /= 2;
                    } else {
                      d[0] += __shfl_xor_sync(0xffffffffu, d[0], o);
                    }
                  }
                  if ((rv & (kCRV / kLCC - 1)) == 0 && c0 + col < ncols)
                    tv[cg + (c0 + col) * kCCG] += (double)d[0];
                }
              }
            }
            if (!ok) return;
            slot ^= 1;
            uu[0] = uu_loc;
            block_reduce<1>(uu, rs, kThreads);
            tv_done = true;
          } else {
          zero_u(Unext);
          __syncthreads();
          phase_a<TX, Acc>(P, Xt, xs_sh, tmem, reinterpret_cast<Acc*>(tpa), j0, wl, vs, red, Ucur + (long long)rep * P.ldn * 8 / (long long)sizeof(Acc));
          double sv1[1] = {sv[0]};
          block_reduce<1>(sv1, rs, ncol);
          if (tid == 0) P.part[((long long)slot * kNF) * G + b] = sv1[0];
          if (!gb.sync()) return;
          // p^T Q p = ||X p||^2 + p^T S p: the partials of p^T S p and the staging
          // of u (with its sum of squares) load together, then one block reduction
          double v2[2] = {tid < G ? ldcg(&P.part[((long long)slot * kNF) * G + tid]) : 0.0,
                          stage_u<Acc>(Ucur, us, n, P.ldn, P.y, false)};
          block_reduce<2>(v2, rs, kThreads);
          slot ^= 1;
          sv[0] = v2[0];
          uu[0] = v2[1];
          }
        } else {
          block_reduce<2>(sv, rs, ncol);
          if (!grid_sum(sv)) return;
          uu[0] = sv[1];
        }
        if (tid == 0) {
          const double pq = uu[0] + sv[0];
          const bool bad = !(pq > 0.0) || !isfinite(pq);
          sc[2] = bad ? 0.0 : rz / pq;
          sc[3] = bad ? (isfinite(pq) ? (double)ST_BREAKDOWN : (double)ST_NONFINITE) : 0.0;
        }
        __syncthreads();
        if (sc[3] != 0.0) { status = (int)sc[3]; break; }
        const double nu = sc[2];
        if constexpr (!IDX) {
          if (!tv_done) phase_c<TX, Acc>(P, Xt, xs_sh, tmem, tred, j0, wl, us, tv);
        } else {
          for (int jj = tid; jj < wl; jj += kThreads) tv[jj] = ps[jj];
        }
        for (int jj = tid; jj < wl; jj += kThreads) {
          const double xn = fma(nu, ps[jj], xs[jj]);
          xs[jj] = xn;
          P.x[j0 + jj] = xn;
          rsm[jj] = fma(-nu, tv[jj] + qs[jj], rsm[jj]);
        }
        __syncthreads();
        apply_precond(P, tri, j0, wl, s_idg, rsm, zs, pw, pw + wp);
        if (two) {
          // 1_c^T r into this iteration's accumulator; clear the previous one (its
          // readers, the p update and the halo of phase A, finished before barrier 1)
          for (int base = warp * 32; base < wl; base += kThreads) {
            const int jj = base + lane;
            warp_add_by_key(Scur, jj < wl ? cid_s[jj] : -1, jj < wl ? rsm[jj] : 0.0);
          }
          for (long long c = j0 + tid; c < j1 && c < nc; c += kThreads) Sold[c] = 0.0;
        }
        double rzn[2] = {0.0, 0.0};
        for (int jj = tid; jj < wl; jj += kThreads) {
          const double rj = rsm[jj];
          rzn[0] = fma(rj, zs[jj], rzn[0]);
          rzn[1] = fma(rj, rj, rzn[1]);
        }
        block_reduce<2>(rzn, rs, ncol);
        if (tid == 0) {
          P.part[((long long)slot * kNF + 0) * G + b] = rzn[0];
          P.part[((long long)slot * kNF + 1) * G + b] = rzn[1];
        }
        if (!gb.sync()) return;
        {
          // the partials of r^T z, r^T r and, with the two-level preconditioner, the
          // component sums for r^T z += sum_c (1_c^T r)^2 / q_c load together; every
          // block reduces them in the same order
          double v3[3] = {0.0, 0.0, 0.0};
          if (tid < G) {
            v3[0] = ldcg(&P.part[((long long)slot * kNF + 0) * G + tid]);
            v3[1] = ldcg(&P.part[((long long)slot * kNF + 1) * G + tid]);
          }
          if (two) {
            for (int c0 = tid; c0 < nc; c0 += 4 * kThreads) {   // 8 loads in flight per thread
              double sv_[4], qv_[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int c = c0 + u * kThreads;
                sv_[u] = c < nc ? ldcg(Scur + c) : 0.0;
                qv_[u] = c < nc ? ldcg(P.qci + c) : 0.0;
                if (c < nc && sc_smem) scs[c] = sv_[u];
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) v3[2] = fma(sv_[u] * sv_[u], qv_[u], v3[2]);
            }
          }
          block_reduce<3>(v3, rs, kThreads);
          slot ^= 1;
          rzn[0] = v3[0] + v3[2];
          rzn[1] = v3[1];
        }
        if (tid == 0) sc[4] = rzn[0] / rz;
        __syncthreads();
        gamma = sc[4];
        rz = rzn[0];
        rr = rzn[1];
        // p_{j+1} = z_j + gamma p_j (shared copy and the other global buffer)
        double* pn = pcur ? P.pb0 : P.pb1;
        for (int jj = tid; jj < wl; jj += kThreads) {
          double zj = zs[jj];
          if (two) {
            const int c = cid_s[jj];
            if (c >= 0) zj = fma(sc_smem ? scs[c] : ldcg(Scur + c), qi_s[jj], zj);
          }
          const double v = fma(gamma, ps[jj], zj);
          ps[jj] = v;
          pn[j0 + jj] = v;
        }
        pcur ^= 1;
        ucur ^= 1;
        ++k;
        __syncthreads();
      }
      cg_total += k;
      cg_mm += k;
      if (status != ST_OK || k == 0 || nref_mm >= P.max_refine) break;
      // ---------------- refinement: r = c - X^T X x - S x in FP64 with this MM
      // iteration's weights.  Accumulator `ucur` is zero here (cleared during
      // the last CG iteration) and receives X x; the other one is cleared.
      void* Ux = ucur ? P.ub1 : P.ub0;
      for (int jj = tid; jj < wl; jj += kThreads) {
        const long long j = j0 + jj;
        const double xj = xs[jj];
        double lap = 0.0;
        if (GK == GK_STENCIL) {
          const unsigned char fl = nb[jj];
          if (fl & NB_L) lap = fma(s_wl[jj], xj - ldcg(P.x + j - 1), lap);
          if (fl & NB_R) lap = fma(s_wr[jj], xj - ldcg(P.x + j + 1), lap);
          if (fl & NB_U) lap = fma(s_wu[jj], xj - ldcg(P.x + j - q2), lap);
          if (fl & NB_D) lap = fma(s_wd[jj], xj - ldcg(P.x + j + q2), lap);
        } else {
          for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e)
            lap = fma(P.wc[e], xj - ldcg(P.x + P.col[e]), lap);
        }
        qs[jj] = fma(s_la[jj], xj, lap);
        vsd[jj] = xj;
      }
      if constexpr (!IDX) {
        zero_u(ucur ? P.ub0 : P.ub1);
        __syncthreads();
        phase_a<TX, double>(P, Xt, xs_sh, tmem, tpa, j0, wl, vsd, redd, reinterpret_cast<double*>(Ux) + (long long)rep * P.ldn);
      }
      if (!gb.sync()) return;
      // the last CG iteration's component sums are no longer read: clear them;
      // the other array was cleared during that iteration and takes 1_c^T r
      double* Slast = ((k - 1 + kpar) & 1) ? P.sc0 : P.sc1;
      double* Snew = ((k - 1 + kpar) & 1) ? P.sc1 : P.sc0;
      if (two)
        for (long long c = j0 + tid; c < j1 && c < nc; c += kThreads) Slast[c] = 0.0;
      if constexpr (!IDX) {
        (void)stage_u<double>(reinterpret_cast<const double*>(Ux), usd, n, P.ldn, P.y, false);
        __syncthreads();
        phase_c<TX, double>(P, Xt, xs_sh, tmem, tred, j0, wl, usd, tv);
      } else {
        for (int jj = tid; jj < wl; jj += kThreads) tv[jj] = xs[jj];
        __syncthreads();
      }
      double rr1[1] = {0.0};
      for (int jj = tid; jj < wl; jj += kThreads) {
        const double rj = (P.c[j0 + jj] - tv[jj]) - qs[jj];
        rsm[jj] = rj;
        rr1[0] = fma(rj, rj, rr1[0]);
      }
      __syncthreads();
      if (two)
        for (int base = warp * 32; base < wl; base += kThreads) {
          const int jj = base + lane;
          warp_add_by_key(Snew, jj < wl ? cid_s[jj] : -1, jj < wl ? rsm[jj] : 0.0);
        }
      block_reduce<1>(rr1, rs, ncol);
      if (!grid_sum(rr1)) return;
      ++nref_mm;
      ++nref_total;
      relres = sqrt(rr1[0]) / P.cnorm;
      if (relres <= sc[5]) {   // accurate: X x stays in accumulator `ucur` for the next MM iteration
        u0_ready = true;
        break;
      }
      kpar = (Snew == P.sc1) ? 1 : 0;   // the restart's k = 0 reads Snew as its start sums
    }
    if (status != ST_OK) break;
    f_prev = f;
    ++mm;
    // x was written before the last grid barrier (or is unchanged): the next
    // reweight may read neighbours' x directly.
    if (cg_mm == 0 && !gb.sync()) return;
  }

  // ---------------- f_eps at the returned iterate (Eq. pert)
  {
    double pe[2] = {0.0, 0.0};
    for (int jj = tid; jj < wl; jj += kThreads) {
      const long long j = j0 + jj;
      const double xj = ldcg(P.x + j);
      const double ax = fabs(xj);
      pe[0] += ax - P.eps * log1p(ax / P.eps);
      if (GK == GK_STENCIL) {
        const unsigned char fl = nb[jj];
        if (fl & NB_R) {
          const double dd = fabs(xj - ldcg(P.x + j + 1));
          pe[1] += dd - P.eps * log1p(dd / P.eps);
        }
        if (fl & NB_D) {
          const double dd = fabs(xj - ldcg(P.x + j + q2));
          pe[1] += dd - P.eps * log1p(dd / P.eps);
        }
      } else {
        for (long long e = P.rowptr[j]; e < P.rowptr[j + 1]; ++e) {
          const long long k = P.col[e];
          if (k > j) {
            const double dd = fabs(xj - ldcg(P.x + k));
            pe[1] += dd - P.eps * log1p(dd / P.eps);
          }
        }
      }
    }
    block_reduce<2>(pe, rs, ncol);
    if (!grid_sum(pe)) return;
    if (b == 0 && tid == 0) {
      DevStats* S = P.stats;
      S->mm_iters = mm;
      S->cg_iters = cg_total;
      S->status = status;
      S->refine_steps = nref_total;
      S->f = f;
      S->f_eps = 0.5 * rss_last + P.lam1 * pe[0] + P.lam2 * pe[1];
      S->rel_change = rel;
      S->cg_relres = relres;
      S->rel_prev = rel_prev;
      S->t0_ns = t_kernel0;
      S->t1_ns = global_ns();
    }
  }
}

// The solve kernel: the body above, with TMEM allocated around it when the
// plan keeps X columns there (tct > 0).  CH selects the chunked one-pass
// Q-apply (x_smem = 1; P.chunked must be set).  Every return of the body comes back
// here, so TMEM is released on every path.  One CTA per SM (launch bounds and
// registers), so the 512-column allocation never waits for another CTA of
// this kernel.
template <typename TX, int GK, bool CH = false>
__global__ void __launch_bounds__(kThreads, 1) mm_solve_kernel(const SolveParams P) {
  __shared__ uint32_t s_tmem;
  const bool use_tmem = P.tct > 0;
  if (use_tmem) {
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&s_tmem, 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  mm_solve_body<TX, GK, CH>(P, use_tmem ? s_tmem : 0u);
  if (use_tmem) {
    tc::fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(s_tmem, 512);
  }
}

}  // namespace flr
