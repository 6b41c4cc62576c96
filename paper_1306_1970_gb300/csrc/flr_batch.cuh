// Batched MM solve: K (lambda1_k, lambda2_k) problems on the same X, y, E in
// one persistent cooperative launch.  Each right-hand side follows the MM
// iteration of Section 3 (reweighting, Eq. lin-sys) with PCG inner solves
// (Algorithm 2); all K run in lockstep and a converged one is masked out.
//
// Per CG iteration the two X contractions of the K Q-applies are GEMMs on
// the tensor cores (tcgen05, FP32 accumulation in TMEM):
//   phase A  U = X P      M = n (128-row tiles), N = K, reduction over p, split
//                         into S chunks per row tile; partial tiles are summed
//   phase C  T = X^T U    M = p (128-column tiles), N = K, reduction over n
// P and U are FP64/FP32 values split into three BF16 slices (hi + mid + lo,
// 24 significant bits), so each product carries FP32-level accuracy.  X is
// BF16 (exact).  The per-RHS vector work (Laplacian, updates, Jacobi
// preconditioner, inner products) is FP64 on the CUDA cores, and every MM
// iteration restarts from an FP64 residual c - X^T X b - S b and objective
// computed on the CUDA cores (FP64 refinement).
//
// Work layout: 128-column tiles are owned round-robin by blocks (tile t by
// block t mod G); a block owns the per-RHS coefficients of its tiles.  Row
// slices of n are reduced block-wise.  Scalar reductions over blocks are FP64
// atomics into rotating slots followed by one grid barrier.
#pragma once
#include "flr_device.cuh"
#include "flr_tc.cuh"

namespace flr {

constexpr int kBT = 256;                 // threads per block
constexpr int kNRMax = 64;               // right-hand sides per launch
constexpr int kTM = 128;                 // tile rows (MMA M); the element loops take 4 x 32 columns
constexpr int kNS = 3;                   // cp.async / MMA pipeline stages
constexpr int kSlices = 3;               // BF16 slices per FP64/FP32 operand
constexpr int kRedSlots = 3;

struct BatchStats {
  int mm_iters, cg_iters, status, refine_steps;
  double f, f_eps, rel_change, cg_relres;
  double rel_prev;             // the relative change of f one MM iteration earlier
};

struct BatchParams {
  const __nv_bfloat16* Xr;     // row-major n x ldp
  const __nv_bfloat16* Xt;     // column-major p x ldn
  long long n, p, ldp, ldn, q2;
  int K, NR;                   // problems; NR = K padded to 32 or 64 (MMA N)
  const double* y;
  const double* c;
  const double* d;
  double cnorm;
  const double* lam1;          // K values (device)
  const double* lam2;
  double eps, tol, tol_cg;
  double tol_cg_rel;           // adaptive inner tolerance factor (0 = off)
  int max_mm, max_cg, min_cg;
  int precond;                 // PC_JACOBI, PC_TRIDIAG or PC_PAPER
  int max_refine;              // FP64 residual restarts of each RHS's inner solve per MM iteration
  int S;                       // split-K chunks per row tile in phase A
  long long kchunk;            // columns per split-K chunk (multiple of 64)
  // per-RHS FP64 state, layout [k][j]
  double *x, *r, *z, *pb0, *pb1, *q, *la, *wl, *wr, *wu, *wd, *idg, *t0;
  double *lmul, *dinv;         // tile tridiagonal LU: multipliers and 1/pivots
  __nv_bfloat16* Ps;           // [3][NR][ldp]
  __nv_bfloat16* Us;           // [3][NR][ldn]
  float* Upart;                // [S][NR][n]
  double* U0part;              // [S][NR][n]
  double* U0;                  // [NR][n]
  double* red;                 // [kRedSlots][4*kNRMax]
  unsigned* bar;
  int* err;
  BatchStats* stats;           // K entries
  long long timeout;
};

__host__ __device__ inline size_t batch_smem_bytes(int NR) {
  const size_t stage = (size_t)kTM * tc::kTileBytesPerRow + (size_t)kSlices * NR * tc::kTileBytesPerRow;
  return kNS * stage                     // operand pipeline
         + (size_t)kNRMax * kTM * 4      // staged accumulator tile (floats)
         + (size_t)64 * kNRMax * 8       // FP64 operand chunk of the refinement passes
         + 32 * (size_t)kNRMax * 8       // per-RHS scalars
         + 256;
}

__device__ __forceinline__ void split3(double v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __double2bfloat16(v);
  const double r1 = v - (double)__bfloat162float(h);
  m = __double2bfloat16(r1);
  const double r2 = r1 - (double)__bfloat162float(m);
  l = __double2bfloat16(r2);
}

// D(tmem, 128 x NR, f32) = A[128 x klen] * (B0 + B1 + B2)[NR x klen]^T
// A row r (r < a_rows, else zero) at A + r*lda + kA0; B slice s row k at
// B + s*bs + k*ldb + kB0.  Columns at or beyond kvalid (relative to the row
// start) are zero.  All threads call; thread 0 issues the MMAs.
struct TcPipe {
  unsigned char* st;     // kNS stages
  uint64_t* mbar;        // kNS mbarriers
  uint32_t phase;        // bit s = parity of stage s's next completion
  uint32_t tmem;
  long long timeout;
  int* err;
};

__device__ __forceinline__ bool tc_tile(TcPipe& tp, const __nv_bfloat16* A, long long lda,
                                        int a_rows, long long kA0, long long a_kvalid,
                                        const __nv_bfloat16* B, long long ldb, long long bs,
                                        long long kB0, long long b_kvalid, long long klen, int NR) {
  using namespace tc;
  const int tid = threadIdx.x;
  const size_t a_bytes = (size_t)kTM * kTileBytesPerRow;
  const size_t b_bytes = (size_t)NR * kTileBytesPerRow;
  const size_t stage_bytes = a_bytes + kSlices * b_bytes;
  const int nch = (int)((klen + KC - 1) / KC);
  const uint32_t idesc = idesc_bf16(kTM, NR);
  auto load = [&](int ch) {
    unsigned char* sb = tp.st + (size_t)(ch % kNS) * stage_bytes;
    const long long k0 = (long long)ch * KC;
    const int a_chunks = kTM * (KC / 8);
    const int b_chunks = kSlices * NR * (KC / 8);
    for (int cidx = tid; cidx < a_chunks + b_chunks; cidx += kBT) {
      if (cidx < a_chunks) {
        const int r = cidx >> 3, kb = cidx & 7;
        const long long kk = kA0 + k0 + kb * 8;
        const bool ok = r < a_rows && (k0 + kb * 8 < klen) && kk + 8 <= a_kvalid;
        const __nv_bfloat16* src = ok ? A + (long long)r * lda + kk : A;
        cp_async16(sb + tile_off(r, kb * 8), src, ok);
      } else {
        const int c2 = cidx - a_chunks;
        const int s = c2 / (NR * 8), rem = c2 % (NR * 8);
        const int r = rem >> 3, kb = rem & 7;
        const long long kk = kB0 + k0 + kb * 8;
        const bool ok = (k0 + kb * 8 < klen) && kk + 8 <= b_kvalid;
        const __nv_bfloat16* src = ok ? B + (long long)s * bs + (long long)r * ldb + kk : B;
        cp_async16(sb + a_bytes + (size_t)s * b_bytes + tile_off(r, kb * 8), src, ok);
      }
    }
  };
  bool ok = true;
  for (int ch = 0; ch < kNS - 1; ++ch) {
    if (ch < nch) load(ch);
    cp_async_commit();
  }
  for (int ch = 0; ch < nch; ++ch) {
    const int nxt = ch + kNS - 1;
    if (nxt < nch) {
      const int s = nxt % kNS;
      if (nxt >= kNS) {   // stage s was last used by chunk nxt - kNS: wait for its MMAs
        if (ok && !mbar_wait(&tp.mbar[s], (tp.phase >> s) & 1u, tp.timeout)) ok = false;
        tp.phase ^= 1u << s;
      }
      load(nxt);
    }
    cp_async_commit();
    cp_async_wait<kNS - 1>();
    fence_async_smem();
    __syncthreads();
    if (tid == 0 && ok) {
      fence_after();
      const unsigned char* sb = tp.st + (size_t)(ch % kNS) * stage_bytes;
      const uint32_t a0 = smem_u32(sb);
      for (int ks = 0; ks < KC / 16; ++ks) {
        for (int s = 0; s < kSlices; ++s) {
          const uint32_t b0 = smem_u32(sb + a_bytes + (size_t)s * b_bytes);
          mma_bf16(tp.tmem, desc(a0 + ks * 2 * kLBO), desc(b0 + ks * 2 * kLBO), idesc,
                   (ch > 0 || ks > 0 || s > 0) ? 1u : 0u);
        }
      }
      commit(&tp.mbar[ch % kNS]);
    }
  }
  // drain: wait for the outstanding commits (the last min(nch, kNS) chunks)
  for (int ch = nch - (nch < kNS ? nch : kNS); ch < nch; ++ch) {
    const int s = ch % kNS;
    if (ok && !mbar_wait(&tp.mbar[s], (tp.phase >> s) & 1u, tp.timeout)) ok = false;
    tp.phase ^= 1u << s;
  }
  fence_after();
  ok = __syncthreads_and(ok ? 1 : 0) != 0;   // one outcome for the whole block
  if (!ok && tid == 0) atomicCAS(tp.err, DERR_NONE, DERR_TIMEOUT);
  return ok;
}

// Copy the 128 x NR accumulator tile out of TMEM into shared memory as
// ts[k][row] (floats).  Warps w and w+4 share TMEM lanes 32(w%4)..+31.
__device__ __forceinline__ void tmem_to_smem(uint32_t tmem, float* ts, int NR) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lane_base = (warp & 3) * 32;
  const int half = NR / 2;
  const int c_begin = (warp < 4) ? 0 : half;
  for (int c0 = c_begin; c0 < c_begin + half; c0 += 16) {
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) ts[(c0 + i) * kTM + lane_base + lane] = v[i];
  }
  tc::fence_before();
  __syncthreads();
}

// Thomas factorisation of the tridiagonal preconditioner of RHS k on the
// 128-column tile starting at j0 (couplings between consecutive columns of the
// tile; block-Jacobi at tile ends, as the single-RHS chunks).  Diagonal:
// lam1 a + lam2 deg (+ X_j^T X_j for PC_TRIDIAG); couplings -lam2 w.
__device__ __forceinline__ void tile_factor(const BatchParams& P, long long k, long long j0, int len) {
  const long long base = k * P.p + j0;
  double prev_d = 1.0, prev_c = 0.0;
  for (int i = 0; i < len; ++i) {
    const long long o = base + i;
    double dd = P.la[o] + ((P.wl[o] + P.wr[o]) + (P.wu[o] + P.wd[o]));
    if (P.precond == PC_TRIDIAG) dd += P.d[j0 + i];
    double m = 0.0;
    if (i > 0) {
      m = -P.wl[o] / prev_d;
      dd = fma(-m, prev_c, dd);
    }
    P.lmul[o] = m;
    P.dinv[o] = 1.0 / dd;
    prev_d = dd;
    prev_c = (i + 1 < len) ? -P.wr[o] : 0.0;
  }
}

// z = M^-1 r on one tile for RHS k with the factors of tile_factor; writes z
// (and p = z when `pz` is given) and returns the tile's sum of r z.  Both
// substitutions are first-order linear
// recurrences, y_i = -m_i y_{i-1} + r_i forward and z_i = a_i z_{i+1} + b_i
// backward (a_i = -c_i / d_i, b_i = y_i / d_i).  Lane l holds entries
// 4l..4l+3, composes their affine maps, a 5-step shuffle scan composes the
// lanes, and each lane then runs its 4 entries from the incoming value.
// All 32 lanes call; lane 0 returns the tile's sum of r z (others: the same).
__device__ __forceinline__ double tile_solve_warp(const BatchParams& P, long long k, long long j0,
                                                  int len, double* pz) {
  const int lane = threadIdx.x & 31;
  const long long base = k * P.p + j0;
  const int i0 = lane * 4;
  double m[4], r[4], a[4], dv[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = i0 + e;
    const bool ok = i < len;
    m[e] = ok ? ldcg(P.lmul + base + i) : 0.0;
    r[e] = ok ? ldcg(P.r + base + i) : 0.0;
    dv[e] = ok ? ldcg(P.dinv + base + i) : 0.0;
    const double c = (ok && i + 1 < len) ? -ldcg(P.wr + base + i) : 0.0;
    a[e] = -c * dv[e];
  }
  // forward: lane map y_out = A y_in + B
  double A = 1.0, B = 0.0;
#pragma unroll
  for (int e = 0; e < 4; ++e) { B = fma(-m[e], B, r[e]); A = -m[e] * A; }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double Ap = __shfl_up_sync(0xffffffffu, A, o);
    const double Bp = __shfl_up_sync(0xffffffffu, B, o);
    if (lane >= o) { B = fma(A, Bp, B); A *= Ap; }
  }
  double y = __shfl_up_sync(0xffffffffu, B, 1);   // y before this lane's entries (y_{-1} = 0)
  if (lane == 0) y = 0.0;
  double b[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) { y = fma(-m[e], y, r[e]); b[e] = y * dv[e]; }
  // backward: lane map z_in(first entry) = A z_out(after last entry) + B
  A = 1.0; B = 0.0;
#pragma unroll
  for (int e = 3; e >= 0; --e) { B = fma(a[e], B, b[e]); A = a[e] * A; }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double An = __shfl_down_sync(0xffffffffu, A, o);
    const double Bn = __shfl_down_sync(0xffffffffu, B, o);
    if (lane + o < 32) { B = fma(A, Bn, B); A *= An; }
  }
  double z = __shfl_down_sync(0xffffffffu, B, 1);   // z after this lane's entries (0 past the tile)
  if (lane == 31) z = 0.0;
  double rz = 0.0;
#pragma unroll
  for (int e = 3; e >= 0; --e) {
    z = fma(a[e], z, b[e]);
    const int i = i0 + e;
    if (i < len) {
      P.z[base + i] = z;
      if (pz) pz[base + i] = z;
      rz = fma(r[e], z, rz);
    }
  }
  return warp_sum(rz);
}

__global__ void __launch_bounds__(kBT, 1) mm_batch_kernel(const BatchParams P) {
  extern __shared__ __align__(1024) unsigned char smb[];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, b = blockIdx.x;
  const long long n = P.n, p = P.p, q2 = P.q2;
  const int K = P.K, NR = P.NR;
  const long long ntiles = (p + kTM - 1) / kTM;
  const long long mtiles = (n + kTM - 1) / kTM;

  const size_t stage_bytes = (size_t)kTM * tc::kTileBytesPerRow + (size_t)kSlices * NR * tc::kTileBytesPerRow;
  unsigned char* stages = smb;
  float* ts = reinterpret_cast<float*>(smb + kNS * stage_bytes);            // [NR][128]
  double* b64 = reinterpret_cast<double*>(ts + kNRMax * kTM);              // [64][kNRMax]
  double* scal = b64 + 64 * kNRMax;                                         // per-RHS scalars
  double* s_rz = scal;                 double* s_rr = scal + kNRMax;
  double* s_nu = scal + 2 * kNRMax;    double* s_gam = scal + 3 * kNRMax;
  double* s_f = scal + 4 * kNRMax;     double* s_fp = scal + 5 * kNRMax;
  double* s_rel = scal + 6 * kNRMax;   double* s_rss = scal + 7 * kNRMax;
  double* s_relres = scal + 8 * kNRMax; double* s_pen = scal + 9 * kNRMax;   // 2 * kNRMax
  double* s_psp = scal + 11 * kNRMax;  double* s_uu = scal + 12 * kNRMax;
  double* s_relp = scal + 13 * kNRMax;
  double* s_tin = scal + 20 * kNRMax;  // inner tolerance of each RHS's current CG cycle
  int* s_act = reinterpret_cast<int*>(scal + 14 * kNRMax);      // MM-active
  int* s_cga = s_act + kNRMax;                                     // CG-active
  int* s_mm = s_act + 2 * kNRMax;
  int* s_cg = s_act + 3 * kNRMax;
  int* s_st = s_act + 4 * kNRMax;
  int* s_rfn = s_act + 5 * kNRMax;                                 // in this refinement round
  int* s_nref = s_act + 6 * kNRMax;                                // refinement rounds, this MM iteration
  int* s_nreft = s_act + 7 * kNRMax;                               // refinement rounds, whole solve
  int* s_cgr = s_act + 8 * kNRMax;                                 // CG iterations, this round
  uint64_t* mbar = reinterpret_cast<uint64_t*>(scal + 32 * kNRMax);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kNS);

  GridBarrier gb{P.bar, P.err, 0u, P.timeout};
  int redi = 0;
  // grid sum of nf fields (per-block partials in `loc` of thread t for field t)
  auto grid_red = [&](double* out, const double* loc_smem, int nf) -> bool {
    double* slot = P.red + (size_t)(redi % kRedSlots) * 4 * kNRMax;
    for (int f = tid; f < nf; f += kBT) atomicAdd(slot + f, loc_smem[f]);
    if (!gb.sync()) return false;
    for (int f = tid; f < nf; f += kBT) out[f] = ldcg(slot + f);
    if (b == 0) {   // zero the slot two reductions ahead (its last reads are done)
      double* z2 = P.red + (size_t)((redi + 2) % kRedSlots) * 4 * kNRMax;
      for (int f = tid; f < 4 * kNRMax; f += kBT) z2[f] = 0.0;
    }
    ++redi;
    __syncthreads();
    return true;
  };

  // ---- TMEM, mbarriers
  if ((tid >> 5) == 0) tc::tmem_alloc(tslot, 64);
  if (tid == 0) {
    for (int s = 0; s < kNS; ++s) tc::mbar_init(&mbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  TcPipe tp{stages, mbar, 0u, tslot[0], P.timeout, P.err};

  // ---- initialisation (Algorithm 1) for every RHS
  for (long long t = b; t < ntiles; t += G)
    for (int e = tid; e < K * kTM; e += kBT) {
      const int k = e / kTM;
      const long long j = t * kTM + (e % kTM);
      if (j < p) P.x[(long long)k * p + j] = P.d[j] != 0.0 ? P.c[j] / P.d[j] : 0.0;
    }
  for (int k = tid; k < kNRMax; k += kBT) {
    s_act[k] = k < K ? 1 : 0; s_cga[k] = 0; s_mm[k] = 0; s_cg[k] = 0; s_st[k] = 0;
    s_rfn[k] = 0; s_nref[k] = 0; s_nreft[k] = 0; s_cgr[k] = 0;
    s_f[k] = 0.0; s_fp[k] = 0.0; s_rel[k] = 0.0; s_relres[k] = 0.0; s_relp[k] = 0.0;
  }
  bool alive = gb.sync();
  int mm = 0, pcur = 0;
  // The per-RHS vector work of a CG iteration is split into units (tile t, RHS k),
  // t-major; block b owns units [u_lo, u_hi), an equal share (the 128-column tiles
  // alone do not divide evenly over the blocks: p = 2e4 gives 157 tiles for 152).
  const long long units = ntiles * (long long)K;
  const long long u_lo = units * b / G, u_hi = units * (b + 1) / G;
  auto is_own = [&](long long j, int k) -> bool {
    const long long u = (j / kTM) * K + k;
    return u >= u_lo && u < u_hi;
  };
  // this block's RHS range [ka, kb) of tile t (empty when ka >= kb)
  auto unit_range = [&](long long t, int& ka, int& kb) {
    const long long a = u_lo > t * K ? u_lo : t * K, e = u_hi < (t + 1) * K ? u_hi : (t + 1) * K;
    ka = (int)(a - t * K);
    kb = (int)(e - t * K);
  };
  // In the tile loops below all 32 lanes of a warp share one RHS index k
  // (128 columns per k, a multiple of 32), so per-RHS sums reduce by warp
  // shuffles and one shared-memory atomic per warp.
  auto wadd = [&](double* dst, double v) {
    v = warp_sum(v);
    if ((tid & 31) == 0 && v != 0.0) atomicAdd(dst, v);
  };

  while (alive) {
    // ---------------- reweight (Eq. lin-sys) per active RHS; S x; penalties
    for (int f = tid; f < 2 * kNRMax; f += kBT) s_pen[f] = 0.0;
    __syncthreads();
    for (long long t = b; t < ntiles; t += G) {
      for (int e = tid; e < K * kTM; e += kBT) {
        const int k = e / kTM;
        if (!s_act[k]) continue;                    // warp-uniform
        const long long j = t * kTM + (e % kTM);
        double v_pen1 = 0.0, v_pen2 = 0.0;
        if (j < p) {
        const double* xk = P.x + (long long)k * p;
        const double xj = ldcg(xk + j);
        const double l1 = P.lam1[k], l2 = P.lam2[k];
        const long long col = j % q2;
        double wl_ = 0.0, wr_ = 0.0, wu_ = 0.0, wd_ = 0.0, lap = 0.0, pen2 = 0.0;
        if (col != 0) { const double v = ldcg(xk + j - 1); wl_ = 1.0 / (fabs(v - xj) + P.eps); lap = fma(wl_, xj - v, lap); }
        if (col != q2 - 1 && j + 1 < p) { const double v = ldcg(xk + j + 1); wr_ = 1.0 / (fabs(xj - v) + P.eps); lap = fma(wr_, xj - v, lap); pen2 += fabs(xj - v); }
        if (j >= q2) { const double v = ldcg(xk + j - q2); wu_ = 1.0 / (fabs(v - xj) + P.eps); lap = fma(wu_, xj - v, lap); }
        if (j + q2 < p) { const double v = ldcg(xk + j + q2); wd_ = 1.0 / (fabs(xj - v) + P.eps); lap = fma(wd_, xj - v, lap); pen2 += fabs(xj - v); }
        const long long o = (long long)k * p + j;
        const double la = l1 / (fabs(xj) + P.eps);
        P.la[o] = la;
        P.wl[o] = l2 * wl_; P.wr[o] = l2 * wr_; P.wu[o] = l2 * wu_; P.wd[o] = l2 * wd_;
        const double deg = (wl_ + wr_) + (wu_ + wd_);
        P.idg[o] = 1.0 / fma(l2, deg, la + P.d[j]);
        P.q[o] = fma(la, xj, l2 * lap);
        v_pen1 = fabs(xj);
        v_pen2 = pen2;
        }
        wadd(&s_pen[k], v_pen1);
        wadd(&s_pen[kNRMax + k], v_pen2);
      }
    }
    if (P.precond != PC_JACOBI) {
      __syncthreads();
      for (long long t = b; t < ntiles; t += G)
        if (tid < K && s_act[tid])
          tile_factor(P, tid, t * kTM, (int)(p - t * kTM < kTM ? p - t * kTM : kTM));
    }
    // ---------------- rounds: first the objective, the outer stop test and the
    // FP64 residual of the new surrogate; then, with max_refine > 0, refinement
    // rounds for the RHS whose CG ran: the true FP64 residual of the same
    // surrogate, and CG restarts from it while it is above tol_cg.
    bool refining = false, finished = false;
    for (int k = tid; k < kNRMax; k += kBT) s_nref[k] = 0;
    __syncthreads();
    while (true) {
    const int* set = refining ? s_rfn : s_act;
    if (refining) {   // S x with this MM iteration's weights (P.q held S p during CG)
      for (long long t = b; t < ntiles; t += G)
        for (int e = tid; e < K * kTM; e += kBT) {
          const int k = e / kTM;
          const long long j = t * kTM + (e % kTM);
          if (!set[k] || j >= p) continue;
          const double* xk = P.x + (long long)k * p;
          const long long o = (long long)k * p + j, col = j % q2;
          const double xj = ldcg(xk + j);
          double lap = 0.0;
          if (col != 0) lap = fma(P.wl[o], xj - ldcg(xk + j - 1), lap);
          if (col != q2 - 1 && j + 1 < p) lap = fma(P.wr[o], xj - ldcg(xk + j + 1), lap);
          if (j >= q2) lap = fma(P.wu[o], xj - ldcg(xk + j - q2), lap);
          if (j + q2 < p) lap = fma(P.wd[o], xj - ldcg(xk + j + q2), lap);
          P.q[o] = fma(P.la[o], xj, lap);
        }
      __syncthreads();
    }
    // u0 = X b and X^T X b recomputed exactly in FP64 on the CUDA cores
    {
      // FP64 refinement pass 1: U0 = X b (CUDA cores, FP64)
      for (long long it = b; it < mtiles * P.S; it += G) {
        const long long mt = it % mtiles, sp = it / mtiles;
        const long long jb = sp * P.kchunk, je = jb + P.kchunk < p ? jb + P.kchunk : p;
        const int row = tid % kTM, h = tid / kTM;       // 2 halves of 32 RHS
        const long long i = mt * kTM + row;
        double acc[32];
        #pragma unroll
        for (int m = 0; m < 32; ++m) acc[m] = 0.0;
        for (long long j0 = jb; j0 < je; j0 += 64) {
          __syncthreads();
          for (int e = tid; e < 64 * kNRMax; e += kBT) {
            const int jj = e / kNRMax, k = e % kNRMax;
            const long long j = j0 + jj;
            b64[jj * kNRMax + k] = (k < K && set[k] && j < je) ? ldcg(P.x + (long long)k * p + j) : 0.0;
          }
          __syncthreads();
          const int jn = (int)(je - j0 < 64 ? je - j0 : 64);
          if (i < n) {
            for (int jj = 0; jj < jn; ++jj) {
              const double xv = (double)__bfloat162float(P.Xt[(j0 + jj) * P.ldn + i]);
              const double* bb = b64 + jj * kNRMax + h * 32;
              #pragma unroll
              for (int m = 0; m < 32; ++m) acc[m] = fma(xv, bb[m], acc[m]);
            }
          }
        }
        if (i < n) {
          #pragma unroll
          for (int m = 0; m < 32; ++m) {
            const int k = h * 32 + m;
            if (k < NR) P.U0part[((long long)sp * NR + k) * n + i] = acc[m];
          }
        }
      }
      __syncthreads();
      if (!refining) {
        if (!grid_red(s_pen, s_pen, 2 * kNRMax)) { alive = false; break; }
      } else if (!gb.sync()) { alive = false; break; }
      // U0 = sum of the split partials, and the residual sum of squares
      for (int f = tid; f < kNRMax; f += kBT) s_rss[f] = 0.0;
      __syncthreads();
      {
        const long long rows_per = (n + G - 1) / G;
        const long long i0 = (long long)b * rows_per, i1 = i0 + rows_per < n ? i0 + rows_per : n;
        for (long long e = tid; e < (long long)K * (i1 > i0 ? i1 - i0 : 0); e += kBT) {
          const int k = (int)(e / (i1 - i0));
          const long long i = i0 + e % (i1 - i0);
          if (!set[k]) continue;
          double sv = 0.0;
          for (int sp = 0; sp < P.S; ++sp) sv += ldcg(P.U0part + ((long long)sp * NR + k) * n + i);
          P.U0[(long long)k * n + i] = sv;
          const double rr = P.y[i] - sv;
          atomicAdd(&s_rss[k], rr * rr);
        }
      }
      __syncthreads();
      if (!refining) {
        if (!grid_red(s_rss, s_rss, kNRMax)) { alive = false; break; }
      } else if (!gb.sync()) { alive = false; break; }
    }
    if (!refining) {
    if (tid < K) {
      const int k = tid;
      if (s_act[k]) {
        const double fk = 0.5 * s_rss[k] + P.lam1[k] * s_pen[k] + P.lam2[k] * s_pen[kNRMax + k];
        s_f[k] = fk;
        if (!isfinite(fk)) { s_act[k] = 0; s_st[k] = ST_NONFINITE; }
        else if (s_mm[k] > 0) {
          s_relp[k] = s_rel[k];
          s_rel[k] = fabs(fk - s_fp[k]) / fabs(s_fp[k]);
          if (s_rel[k] <= P.tol) s_act[k] = 0;
        }
        if (s_act[k] && s_mm[k] >= P.max_mm) { s_act[k] = 0; s_st[k] = ST_NOTCONV; }
      }
    }
    __syncthreads();
    int nact = 0;
    for (int k = 0; k < K; ++k) nact += s_act[k];
    if (nact == 0) { finished = true; break; }
    }
    // ---------------- FP64 refinement pass 2: r0 = c - X^T U0 - S b; z0; p1 = z0
    for (int f = tid; f < kNRMax; f += kBT) { s_rz[f] = 0.0; s_rr[f] = 0.0; }
    __syncthreads();
    for (long long t = b; t < ntiles; t += G) {
      const int cl = tid % kTM, h = tid / kTM;
      const long long j = t * kTM + cl;
      double acc[32];
#pragma unroll
      for (int m = 0; m < 32; ++m) acc[m] = 0.0;
      for (long long i0 = 0; i0 < n; i0 += 64) {
        __syncthreads();
        for (int e = tid; e < 64 * kNRMax; e += kBT) {
          const int ii = e / kNRMax, k = e % kNRMax;
          const long long i = i0 + ii;
          b64[ii * kNRMax + k] = (k < K && set[k] && i < n) ? ldcg(P.U0 + (long long)k * n + i) : 0.0;
        }
        __syncthreads();
        const int in = (int)(n - i0 < 64 ? n - i0 : 64);
        if (j < p) {
          for (int ii = 0; ii < in; ++ii) {
            const double xv = (double)__bfloat162float(P.Xt[j * P.ldn + i0 + ii]);
            const double* bb = b64 + ii * kNRMax + h * 32;
#pragma unroll
            for (int m = 0; m < 32; ++m) acc[m] = fma(xv, bb[m], acc[m]);
          }
        }
      }
      if (j < p) {
#pragma unroll
        for (int m = 0; m < 32; ++m) {
          const int k = h * 32 + m;
          if (k < K && set[k]) P.t0[(long long)k * p + j] = acc[m];
        }
      }
    }
    __syncthreads();
    {
      double* pc = pcur ? P.pb1 : P.pb0;
      for (long long t = b; t < ntiles; t += G) {
        for (int e = tid; e < K * kTM; e += kBT) {
          const int k = e / kTM;
          const long long j = t * kTM + (e % kTM);
          if (!set[k]) continue;                    // warp-uniform
          double v_rz = 0.0, v_rr = 0.0;
          if (j < p) {
            const long long o = (long long)k * p + j;
            const double rj = (P.c[j] - P.t0[o]) - P.q[o];
            P.r[o] = rj;
            v_rr = rj * rj;
            if (P.precond == PC_JACOBI) {
              const double zj = rj * P.idg[o];
              P.z[o] = zj; pc[o] = zj;
              v_rz = rj * zj;
            }
          }
          if (P.precond == PC_JACOBI) wadd(&s_rz[k], v_rz);
          wadd(&s_rr[k], v_rr);
        }
        if (P.precond != PC_JACOBI) {
          __syncthreads();
          const int len = (int)(p - t * kTM < kTM ? p - t * kTM : kTM);
          for (int k = tid >> 5; k < K; k += kBT / 32)   // one warp per RHS
            if (set[k]) {
              const double rz = tile_solve_warp(P, k, t * kTM, len, pc);
              if ((tid & 31) == 0) atomicAdd(&s_rz[k], rz);
            }
          __syncthreads();
        }
      }
    }
    __syncthreads();
    // rz and rr as one 2*kNRMax-field reduction
    {
      double* tmp = s_nu;   // s_nu, s_gam are adjacent: 2*kNRMax doubles
      for (int f = tid; f < kNRMax; f += kBT) { tmp[f] = s_rz[f]; tmp[kNRMax + f] = s_rr[f]; }
      __syncthreads();
      if (!grid_red(tmp, tmp, 2 * kNRMax)) { alive = false; break; }
      for (int f = tid; f < kNRMax; f += kBT) { s_rz[f] = tmp[f]; s_rr[f] = tmp[kNRMax + f]; s_gam[f] = 0.0; }
    }
    if (tid < kNRMax) {
      const int k = tid;
      int go = (k < K && set[k] && s_act[k]) ? 1 : 0;
      const double rel_r = go ? sqrt(s_rr[k]) / P.cnorm : 0.0;
      if (refining && go) {   // the true residual decides whether CG restarts
        ++s_nref[k];
        ++s_nreft[k];
        s_relres[k] = rel_r;
        if (rel_r <= s_tin[k]) go = 0;
      }
      // the cycle's inner tolerance: tol_cg, or with tol_cg_rel = theta > 0,
      // max(tol_cg, min(theta * rel_change, ||r0|| / (2 ||c||))) as in flr_solve
      if (go) {
        const double ad = P.tol_cg_rel * (s_mm[k] > 0 ? s_rel[k] : 1.0);
        s_tin[k] = P.tol_cg_rel > 0.0 ? fmax(P.tol_cg, fmin(ad, 0.5 * rel_r)) : P.tol_cg;
      }
      s_cga[k] = go;
      s_cgr[k] = 0;
    }
    __syncthreads();
    // ---------------- CG iterations for all active RHS
    int kcg = 0;
    while (true) {
      if (tid < K) {
        const int k = tid;
        if (s_cga[k]) {
          const double rel_r = sqrt(s_rr[k]) / P.cnorm;
          s_relres[k] = rel_r;
          if (kcg >= P.max_cg || (kcg >= P.min_cg && rel_r <= s_tin[k])) s_cga[k] = 0;
          else { s_cg[k] += 1; s_cgr[k] += 1; }
        }
      }
      __syncthreads();
      int ncga = 0;
      for (int k = 0; k < K; ++k) ncga += s_cga[k];
      if (ncga == 0) break;
      const double* pc = pcur ? P.pb1 : P.pb0;
      const double* po = pcur ? P.pb0 : P.pb1;
      // (a) S p, p^T S p, and the BF16 slices of p for this block's units
      for (int f = tid; f < kNRMax; f += kBT) s_psp[f] = 0.0;
      __syncthreads();
      // this block's units: warp w takes RHS k = ka + w, ka + w + 8, ...; lane l
      // the columns l + 32u of the tile, u = 0..3, with every load of the four
      // issued before their use.  Rows k >= K of the P slices stay zero.
      for (long long t = u_lo / K; t < ntiles && t * K < u_hi; ++t) {
        int ka, kb;
        unit_range(t, ka, kb);
        for (int k = ka + warp; k < kb; k += kBT / 32) {
          const bool act = s_cga[k];              // warp-uniform
          const double g = act ? s_gam[k] : 0.0;
          const long long ko = (long long)k * p;
          auto pv = [&](long long kk) -> double {
            if (kcg == 0 || is_own(kk, k)) return ldcg(pc + ko + kk);
            return fma(g, ldcg(po + ko + kk), ldcg(P.z + ko + kk));
          };
          double pj[4], la[4], wl[4], wr[4], wu[4], wd[4], nl[4], nr[4], nu[4], nd[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const long long j = t * kTM + lane + 32 * u;
            const bool ok = act && j < p;
            const long long o = ko + j;
            const long long col = j % q2;
            pj[u] = ok ? ldcg(pc + o) : 0.0;
            la[u] = ok ? ldcg(P.la + o) : 0.0;
            wl[u] = ok ? ldcg(P.wl + o) : 0.0;
            wr[u] = ok ? ldcg(P.wr + o) : 0.0;
            wu[u] = ok ? ldcg(P.wu + o) : 0.0;
            wd[u] = ok ? ldcg(P.wd + o) : 0.0;
            nl[u] = (ok && col != 0) ? pv(j - 1) : 0.0;
            nr[u] = (ok && col != q2 - 1 && j + 1 < p) ? pv(j + 1) : 0.0;
            nu[u] = (ok && j >= q2) ? pv(j - q2) : 0.0;
            nd[u] = (ok && j + q2 < p) ? pv(j + q2) : 0.0;
          }
          double v_psp = 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const long long j = t * kTM + lane + 32 * u;
            __nv_bfloat16 h = __float2bfloat16(0.f), m = h, l = h;
            if (act && j < p) {
              const long long col = j % q2;
              double lap = 0.0;
              if (col != 0) lap = fma(wl[u], pj[u] - nl[u], lap);
              if (col != q2 - 1 && j + 1 < p) lap = fma(wr[u], pj[u] - nr[u], lap);
              if (j >= q2) lap = fma(wu[u], pj[u] - nu[u], lap);
              if (j + q2 < p) lap = fma(wd[u], pj[u] - nd[u], lap);
              const double spj = fma(la[u], pj[u], lap);
              P.q[ko + j] = spj;
              v_psp = fma(pj[u], spj, v_psp);
              split3(pj[u], h, m, l);
            }
            if (j < p) {
              P.Ps[(0LL * NR + k) * P.ldp + j] = h;
              P.Ps[(1LL * NR + k) * P.ldp + j] = m;
              P.Ps[(2LL * NR + k) * P.ldp + j] = l;
            }
          }
          wadd(&s_psp[k], v_psp);
        }
      }
      __syncthreads();
      if (!grid_red(s_psp, s_psp, kNRMax)) { alive = false; break; }
      // (b) phase A: U partials = X[rows, chunk] P[chunk]  (tensor cores)
      for (long long it = b; it < mtiles * P.S; it += G) {
        const long long mt = it % mtiles, sp = it / mtiles;
        const long long jb = sp * P.kchunk;
        const long long klen = jb + P.kchunk < P.ldp ? P.kchunk : P.ldp - jb;
        if (klen <= 0) continue;
        const int rows = (int)(n - mt * kTM < kTM ? n - mt * kTM : kTM);
        if (!tc_tile(tp, P.Xr + mt * kTM * P.ldp, P.ldp, rows, jb, P.ldp, P.Ps, P.ldp,
                     (long long)NR * P.ldp, jb, P.ldp, klen, NR)) { alive = false; break; }
        tmem_to_smem(tp.tmem, ts, NR);
        for (int e = tid; e < NR * kTM; e += kBT) {
          const int k = e / kTM, rr = e % kTM;
          const long long i = mt * kTM + rr;
          if (i < n) P.Upart[((long long)sp * NR + k) * n + i] = ts[k * kTM + rr];
        }
        __syncthreads();
      }
      if (!alive) break;
      if (!gb.sync()) { alive = false; break; }
      // (c) U = sum of partials; ||U_k||^2; BF16 slices of U
      for (int f = tid; f < kNRMax; f += kBT) s_uu[f] = 0.0;
      __syncthreads();
      {
        const long long rows_per = (P.ldn + G - 1) / G;
        const long long i0 = (long long)b * rows_per;
        const long long i1 = i0 + rows_per < P.ldn ? i0 + rows_per : P.ldn;
        const long long cnt = i1 > i0 ? i1 - i0 : 0;
        for (long long e = tid; e < (long long)NR * cnt; e += kBT) {
          const int k = (int)(e / cnt);
          const long long i = i0 + e % cnt;
          double s = 0.0;
          if (i < n && k < K && s_cga[k])
            for (int sp = 0; sp < P.S; ++sp) s += (double)ldcg(P.Upart + ((long long)sp * NR + k) * n + i);
          __nv_bfloat16 h, m, l;
          split3(s, h, m, l);
          P.Us[(0LL * NR + k) * P.ldn + i] = h;
          P.Us[(1LL * NR + k) * P.ldn + i] = m;
          P.Us[(2LL * NR + k) * P.ldn + i] = l;
          if (s != 0.0) atomicAdd(&s_uu[k], s * s);
        }
      }
      __syncthreads();
      if (!grid_red(s_uu, s_uu, kNRMax)) { alive = false; break; }
      if (tid < K) {
        const int k = tid;
        double nu = 0.0;
        if (s_cga[k]) {
          const double pq = s_uu[k] + s_psp[k];
          if (!(pq > 0.0) || !isfinite(pq)) {
            s_cga[k] = 0; s_act[k] = 0; s_st[k] = isfinite(pq) ? ST_BREAKDOWN : ST_NONFINITE;
          } else {
            nu = s_rz[k] / pq;
          }
        }
        s_nu[k] = nu;
      }
      __syncthreads();
      // (d) phase C: T = X^T U for this block's units (tensor cores), then the updates
      double* loc = s_pen;   // 2*kNRMax partials: r^T z, r^T r
      for (int f = tid; f < 2 * kNRMax; f += kBT) loc[f] = 0.0;
      __syncthreads();
      // this block's units: T for tile t and RHS rows [kq, kq + nq) of U (nq = 32
      // or 64, covering [ka, kb) and staying inside the NR rows), then the updates
      for (long long t = u_lo / K; t < ntiles && t * K < u_hi; ++t) {
        int ka, kb;
        unit_range(t, ka, kb);
        if (ka >= kb) continue;
        const int nq = (kb - ka <= 32 || NR == 32) ? 32 : 64;
        const int kq = ka + nq <= NR ? ka : NR - nq;
        const int rows = (int)(p - t * kTM < kTM ? p - t * kTM : kTM);
        if (!tc_tile(tp, P.Xt + t * kTM * P.ldn, P.ldn, rows, 0, P.ldn, P.Us + (long long)kq * P.ldn, P.ldn,
                     (long long)NR * P.ldn, 0, P.ldn, P.ldn, nq)) { alive = false; break; }
        tmem_to_smem(tp.tmem, ts, nq);
        const bool jac = P.precond == PC_JACOBI;
        for (int k = ka + warp; k < kb; k += kBT / 32) {   // as in (a): warp per RHS, 4 columns per lane
          if (!s_cga[k]) continue;                  // warp-uniform
          const double nu = s_nu[k];
          const long long ko = (long long)k * p;
          double qv[4], pv4[4], xv[4], rv[4], iv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const long long j = t * kTM + lane + 32 * u;
            const bool ok = j < p;
            const long long o = ko + j;
            qv[u] = ok ? ldcg(P.q + o) : 0.0;
            pv4[u] = ok ? ldcg(pc + o) : 0.0;
            xv[u] = ok ? ldcg(P.x + o) : 0.0;
            rv[u] = ok ? ldcg(P.r + o) : 0.0;
            iv[u] = (ok && jac) ? ldcg(P.idg + o) : 0.0;
          }
          double v_rz = 0.0, v_rr = 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int cl = lane + 32 * u;
            const long long j = t * kTM + cl;
            if (j < p) {
              const long long o = ko + j;
              const double tj = (double)ts[(k - kq) * kTM + cl];
              const double qj = tj + qv[u];
              P.x[o] = fma(nu, pv4[u], xv[u]);
              const double rj = fma(-nu, qj, rv[u]);
              P.r[o] = rj;
              v_rr = fma(rj, rj, v_rr);
              if (jac) {
                const double zj = rj * iv[u];
                P.z[o] = zj;
                v_rz = fma(rj, zj, v_rz);
              }
            }
          }
          if (jac) wadd(&loc[k], v_rz);
          wadd(&loc[kNRMax + k], v_rr);
        }
        __syncthreads();
        if (P.precond != PC_JACOBI) {
          for (int k = ka + (tid >> 5); k < kb; k += kBT / 32)   // one warp per RHS
            if (s_cga[k]) {
              const double rz = tile_solve_warp(P, k, t * kTM, rows, nullptr);
              if ((tid & 31) == 0) atomicAdd(&loc[k], rz);
            }
          __syncthreads();
        }
      }
      if (!alive) break;
      if (!grid_red(loc, loc, 2 * kNRMax)) { alive = false; break; }
      // (e) gamma_k and p_{j+1} = z + gamma p
      if (tid < K) {
        const int k = tid;
        if (s_cga[k]) {
          s_gam[k] = loc[k] / s_rz[k];
          s_rz[k] = loc[k];
          s_rr[k] = loc[kNRMax + k];
        }
      }
      __syncthreads();
      {
        double* pn = pcur ? P.pb0 : P.pb1;
        for (long long t = u_lo / K; t < ntiles && t * K < u_hi; ++t) {
          int ka, kb;
          unit_range(t, ka, kb);
          for (int k = ka + warp; k < kb; k += kBT / 32) {
            if (!s_cga[k]) continue;                // warp-uniform
            const double g = s_gam[k];
            const long long ko = (long long)k * p;
            double pv4[4], zv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const long long j = t * kTM + lane + 32 * u;
              pv4[u] = j < p ? ldcg(pc + ko + j) : 0.0;
              zv[u] = j < p ? ldcg(P.z + ko + j) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const long long j = t * kTM + lane + 32 * u;
              if (j < p) pn[ko + j] = fma(g, pv4[u], zv[u]);
            }
          }
        }
      }
      pcur ^= 1;
      ++kcg;
      __syncthreads();
    }
    if (!alive) break;
    // the next refinement round: RHS whose CG ran in this round, with restarts left
    if (tid < kNRMax) {
      const int k = tid;
      s_rfn[k] = (k < K && s_act[k] && s_cgr[k] > 0 && s_nref[k] < P.max_refine) ? 1 : 0;
    }
    __syncthreads();
    int nrf = 0;
    for (int k = 0; k < K; ++k) nrf += s_rfn[k];
    if (nrf == 0) break;
    refining = true;
    }   // rounds
    if (finished) break;

    if (!alive) break;
    if (tid < K) {
      if (s_act[tid]) { s_fp[tid] = s_f[tid]; s_mm[tid] += 1; }
    }
    ++mm;
    __syncthreads();
    if (!gb.sync()) { alive = false; break; }
  }

  // ---- statistics (f_eps is left to the host)
  if (alive && b == 0) {
    for (int k = tid; k < K; k += kBT) {
      BatchStats* S = P.stats + k;
      S->mm_iters = s_mm[k];
      S->cg_iters = s_cg[k];
      S->status = s_st[k];
      S->refine_steps = s_nreft[k];
      S->f = s_f[k];
      S->f_eps = 0.0;
      S->rel_change = s_rel[k];
      S->cg_relres = s_relres[k];
      S->rel_prev = s_relp[k];
    }
  }
  tc::fence_before();
  __syncthreads();
  if ((tid >> 5) == 0) tc::tmem_dealloc(tslot[0], 64);
}

}  // namespace flr
