// Device-side building blocks of the FLR solver: X-element traits, streaming
// loads, a bounded grid barrier, deterministic block reductions.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace flr {

constexpr int kThreads = 256;            // threads per block of the solve kernel
constexpr int kWarps = kThreads / 32;
constexpr int kNF = 4;                   // scalar fields per grid-reduction slot
constexpr int kMaxLevels = 13;           // PCR levels: block chunks up to 8192 indices

enum DevErr : int { DERR_NONE = 0, DERR_TIMEOUT = 1 };

// ---------------------------------------------------------------------------
// X element traits: V elements per 16-byte vector, accumulator type Acc.
// ---------------------------------------------------------------------------
template <typename TX> struct XT;

// X is re-read every CG iteration: its loads skip L1 and carry an L2
// evict_last policy, so other traffic (an L2 flush, the vectors) evicts X last.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// Bring the L2 line holding p in ahead of its load (evict_last, as the loads),
// without holding a register: more of X in flight from HBM per thread.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2::evict_last [%0];" :: "l"(p));
}
__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p), "l"(l2_keep_policy()));
  return r;
}

template <> struct XT<double> {
  static constexpr int V = 2;
  using Acc = double;
  __device__ static __forceinline__ void cvt(const uint4& v, double (&o)[2]) {
    o[0] = __hiloint2double((int)v.y, (int)v.x);
    o[1] = __hiloint2double((int)v.w, (int)v.z);
  }
};
template <> struct XT<float> {
  static constexpr int V = 4;
  using Acc = float;
  __device__ static __forceinline__ void cvt(const uint4& v, float (&o)[4]) {
    o[0] = __uint_as_float(v.x); o[1] = __uint_as_float(v.y);
    o[2] = __uint_as_float(v.z); o[3] = __uint_as_float(v.w);
  }
};
template <> struct XT<__nv_bfloat16> {
  static constexpr int V = 8;
  using Acc = float;
  __device__ static __forceinline__ void cvt(const uint4& v, float (&o)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // bf16 -> f32 is a 16-bit shift, exact
      o[2 * i] = __uint_as_float(w[i] << 16);
      o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};
template <> struct XT<__half> {
  static constexpr int V = 8;
  using Acc = float;
  __device__ static __forceinline__ void cvt(const uint4& v, float (&o)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
      float2 f = __half22float2(h);
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
};

// X = I (the FLSA): no matrix is stored or read; the solve kernel replaces
// every X product by the vector itself.  V and Acc only size shared buffers.
struct IdX {};
template <> struct XT<IdX> {
  static constexpr int V = 2;
  using Acc = double;
};

// Device-wide nanosecond timer (comparable across kernels on one GPU).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// coherent (L2) loads for data other blocks wrote during this launch
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Grid barrier for a cooperative launch.  `counter` is zeroed by the host
// before the launch; barrier number e (1-based) completes when the counter
// reaches e * gridDim.x.  Every wait is bounded: after `timeout` clock
// cycles the block records DERR_TIMEOUT in *err and returns false, and a
// block that sees *err set returns false too, so all blocks leave.
// ---------------------------------------------------------------------------
struct GridBarrier {
  unsigned* counter;
  int* err;
  unsigned epoch;
  long long timeout;

  __device__ __forceinline__ bool sync() {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      epoch += 1;
      const unsigned target = epoch * gridDim.x;
      // the block's writes (ordered before this thread by __syncthreads) are
      // released to the GPU scope, then the arrival is counted
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
      int ok = 1;
      const long long t0 = clock64();
      unsigned spins = 0;
      while (true) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
        if ((int)(v - target) >= 0) break;
        if (*((volatile int*)err) != DERR_NONE) { ok = 0; break; }
        if (++spins > 32) {
          __nanosleep(32);
          if (clock64() - t0 > timeout) {
            atomicCAS(err, DERR_NONE, DERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
      s_ok = ok;   // the acquire loads above order the reads that follow the barrier
    }
    __syncthreads();
    return s_ok != 0;
  }
};

// ---------------------------------------------------------------------------
// Split grid barrier: arrive(s) and wait(s) for s = 0, 1, 2, ... in order, with
// at most one barrier outstanding between a block's arrive(s + 1) and its
// wait(s).  Barrier s counts on counter s & 1 (two counters 128 bytes apart,
// zeroed by the host before the launch), so a block that arrives at s + 1
// before others arrive at s cannot complete barrier s early.  Waits are
// bounded as in GridBarrier.
// ---------------------------------------------------------------------------
struct SplitBarrier {
  unsigned* cnt;
  int* err;
  unsigned epoch[2];
  long long timeout;

  __device__ __forceinline__ void arrive(int s) {
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(cnt + 32 * (s & 1)) : "memory");
    }
  }
  __device__ __forceinline__ bool wait(int s) {
    __shared__ int s_ok2;
    const int c = s & 1;
    epoch[c] += 1;
    if (threadIdx.x == 0) {
      const unsigned target = epoch[c] * gridDim.x;
      const unsigned* ctr = cnt + 32 * c;
      int ok = 1;
      const long long t0 = clock64();
      unsigned spins = 0;
      while (true) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if ((int)(v - target) >= 0) break;
        if (*((volatile int*)err) != DERR_NONE) { ok = 0; break; }
        if (++spins > 32) {
          __nanosleep(32);
          if (clock64() - t0 > timeout) {
            atomicCAS(err, DERR_NONE, DERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
      s_ok2 = ok;
    }
    __syncthreads();
    return s_ok2 != 0;
  }
};

// ---------------------------------------------------------------------------
// Deterministic warp reduction (fixed shuffle pattern).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace flr
