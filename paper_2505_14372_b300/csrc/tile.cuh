// Shared-memory resident 2-D FFT tile for one N x N complex64 wavefield.
//
// One wavefield lives in the shared memory of a cluster of G CTAs (G = 1 for
// N <= 128; G = 2 for 192; G = 4 for 256, because 192^2 and 256^2 complex64
// waves exceed one SM's 227 KB).  Every 1-D transform is split N = R1 * R2
// (R2 = 16):
//   forward:  strided stage   (R1-point DFT over elements n2 + R2*n1, then
//                              twiddle W_N^(n2 k1)),
//             contiguous stage (R2-point DFT over the R2 consecutive slots of
//                              group k1); the spectrum is left in digit-
//                              permuted order: slot k2 + R2*k1 holds bin
//                              k1 + R1*k2.
//   inverse:  contiguous stage (inverse R2-point DFT, twiddle W_N^-(n2 k1)),
//             strided stage   (inverse R1-point DFT), natural order out.
// All stages are in place, so FFT -> pointwise product -> inverse FFT (one
// multislice propagation) never reorders data, and the pointwise ops are
// fused into the stages that touch the data anyway.
//
// Layouts (per CTA of rank c): the smem holds G blocks of ROWS x ROWS
// (ROWS = N/G).  Row layout: block b = (my rows) x (columns of CTA b).
// Column layout: block b = (rows of CTA b) x (my columns).  Switching layout
// is a block transpose across the cluster: element (CTA c, block b, row r,
// column cc) moves to (CTA b, block c, r, cc); it is fused into the last
// stage of a row pass (row -> column) and of an inverse column pass (column
// -> row).  For G = 2 that stage writes its results in place and every
// warp sends the off-diagonal slots it has just finished (the same swizzle
// in both CTAs) to the partner's idle buffer as bulk shared::cluster
// copies, so the transfer overlaps the rest of the stage; the copies count
// their bytes on the partner's mbarrier (no cluster barrier per switch).
// Between the two row stages no data crosses rows, so for G = 2 groups of
// warps that own whole rows meet at their own named barriers there.
// G = 4 stages the block in registers and writes it with
// st.shared::cluster between two cluster barriers.
//
// Bank conflicts: slot (b, r, cc) sits at base(b) + r*ROWS +
// 2((cc >> 1) ^ f) + (cc & 1) with f = (R1 r + cc / R2 + o) mod 8: the XOR
// permutes 16-byte column pairs, so columns cc, cc+1 (cc even) stay adjacent
// and in order.  o = NB b (NB = ROWS / R2) for G = 1, 4; for G = 2, o = 6 on
// the off-diagonal block and 4 * rank on the diagonal one.  The strided and
// column stages walk 16 consecutive cc of one row with 8-byte accesses (f
// constant: 16 distinct bank pairs per half-warp); the row-contiguous stage
// reads and writes its 16 consecutive columns as 8 16-byte pairs, and the 8
// lanes (r, k1) of a quarter-warp (a run of 8 consecutive k1 mod R1) get 8
// distinct f, so they hit 8 distinct 16-byte bank groups.
#pragma once
#include <stdint.h>

#include "check.cuh"
#include "radix.cuh"

namespace ptycho {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster_s32(uint32_t addr, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// Arrive without ordering memory: used where the partner only needs to know
// that this CTA has consumed (loaded into registers) the slots it will
// overwrite.
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// fire-and-forget vector reduction into global memory (sm_90+)
__device__ __forceinline__ void red_add(float2* p, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

// ---- mbarrier-signalled exchange between the two CTAs of a 192x192 tile --
// A layout switch copies the off-diagonal block into the partner's idle
// buffer with bulk copies that count their bytes on the partner's mbarrier;
// the partner waits on that mbarrier (expected bytes = one block) instead of
// both CTAs meeting at a cluster barrier.  Reuse of a buffer is ordered by
// the data flow: a CTA copies into its partner's buffer only after it has
// received the partner's data of the opposite switch, which the partner
// sends (from that very buffer) after its last write to it, and whose
// arrival means the copy engine has finished reading it.
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ uint64_t mbar_arrive(uint32_t bar) {
  uint64_t st;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(bar) : "memory");
  return st;
}
__device__ __forceinline__ uint64_t mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  uint64_t st;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;" : "=l"(st) : "r"(bar), "r"(bytes) : "memory");
  return st;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint64_t st) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "l"(st)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void st_cluster2(uint32_t addr, float2 a, float2 b) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a.x), "f"(a.y), "f"(b.x),
               "f"(b.y)
               : "memory");
}
// exchange waits that gave up (bounded wait); read and cleared by the host
static __device__ unsigned g_exchange_timeouts;
constexpr unsigned kExchangeSpin = 1u << 22;

struct NoLoad {
  __device__ float2 operator()(int, int) const { return make_float2(0.f, 0.f); }
};
struct NoOp {
  __device__ void operator()(int, int, float2&) const {}
};
struct NoPre {
  struct type {};
  __device__ type operator()(int, int) const { return {}; }
};
struct NoOp4 {
  template <class P>
  __device__ void operator()(int, int, float2&, const P&) const {}
};

template <int N_, int G_, int R2_, int T_, int MINB_ = 1>
struct Tile {
  static constexpr int N = N_, G = G_, R2 = R2_, R1 = N_ / R2_, T = T_, MINB = MINB_;
  static constexpr int NP = N * N;
  static constexpr int ROWS = N / G;
  static constexpr int NB = ROWS / R2;               // R2-groups per block row
  static constexpr int BLK = ROWS * ROWS;
  // G == 2: the off-diagonal block is double-buffered (XA holds it in the
  // row layout, XB in the column layout), so a layout switch writes into the
  // partner's idle buffer and needs one cluster barrier and no register
  // staging.  G == 4 keeps one slot per block and stages in registers.
  static constexpr bool XB = (G == 2);
  static constexpr int WAVE = XB ? 3 * BLK : G * BLK;  // float2 slots per CTA
  static constexpr int TS = ROWS * R2;               // strided-stage tasks (R1 elements)
  static constexpr int TC = ROWS * R1;               // contiguous-stage tasks (R2 elements)
  static constexpr int SPT = (TS + T - 1) / T;       // strided tasks per thread (last may idle)
  static constexpr int CPT = (TC + T - 1) / T;       // contiguous tasks per thread
  // smem: wave, twS[N], twC[N], rampY[N], rampX[N], chirp[2][N], fsq[N] (int),
  // then (G == 2) the two exchange mbarriers: [0] row-layout block arrived,
  // [1] column-layout block arrived
  static constexpr size_t BAR_OFF = sizeof(float2) * (WAVE + 6 * N) + sizeof(int) * N;
  static constexpr size_t SMEM = BAR_OFF + (XB ? 16 : 0);
  static_assert(BAR_OFF % 8 == 0, "mbarrier alignment");
  static_assert(N == R1 * R2 && R2 % 16 == 0, "N = R1 R2 with R2 a multiple of 16");
  static_assert(N % G == 0 && ROWS % R2 == 0 && ROWS % 16 == 0, "block split");
  static_assert(T % 32 == 0, "whole warps");
  static_assert(!XB || (TC % T == 0 && TS % T == 0 && ROWS % 32 == 0 && NB * 2 == R1),
                "2-CTA exchange: whole rounds, warps of 32 consecutive columns");

  // Row stages: NG groups of GT threads, group g owning rows
  // [RG g, RG (g + 1)) in both row stages, so the barriers between them (no
  // data crosses rows) are per group, named barrier 1 + g.
  static constexpr int NG = 4, GT = T / NG, RG = ROWS / NG;
  static constexpr bool ROWG = T % NG == 0 && GT % 32 == 0 && GT % R1 == 0 && GT % R2 == 0 && ROWS % NG == 0 &&
                               (RG * R1) % GT == 0 && (RG * R2) % GT == 0;
  // id of this thread's task in round t of a row stage, tasks enumerated
  // row-major with PER tasks per row
  template <int PER>
  __device__ static __forceinline__ int row_task(int t) {
    if constexpr (ROWG) return RG * PER * (int)(threadIdx.x / GT) + (int)(threadIdx.x % GT) + GT * t;
    else return (int)threadIdx.x + T * t;
  }
  // barrier between two row stages
  __device__ static void row_sync() {
    if constexpr (ROWG) asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / GT)), "r"(GT) : "memory");
    else __syncthreads();
  }

  // natural DFT bin held by spectral slot p, and slot of natural bin n
  __host__ __device__ static constexpr int nat(int p) { return p / R2 + R1 * (p % R2); }
  __host__ __device__ static constexpr int perm(int n) { return n / R1 + R2 * (n % R1); }
  // signed DFT frequency (fftfreq order) of natural bin n
  __host__ __device__ static constexpr int freq(int n) { return n < (N + 1) / 2 ? n : n - N; }

  // swizzled slot of (logical block b, row r, column cc) within one CTA, in
  // the row layout (COL = false) or the column layout (COL = true)
  template <bool COL>
  __device__ static __forceinline__ int slot(int rank, int b, int r, int cc) {
    int base, f;
    if constexpr (XB) {
      // the off-diagonal block has the same swizzle in both CTAs and both
      // layouts, so a layout switch moves it as one contiguous bulk copy
      const bool diag = b == rank;
      base = diag ? 0 : (COL ? 2 * BLK : BLK);
      f = (R1 * r + cc / R2 + (diag ? 4 * rank : 6)) & 7;
    } else {
      base = G == 1 ? 0 : b * BLK;
      f = (R1 * r + NB * b + cc / R2) & 7;
    }
    const int idx = base + r * ROWS + (((cc >> 1) ^ f) << 1) + (cc & 1);
    return chk(idx >= 0 && idx < WAVE, kChkSmem) ? idx : 0;
  }
  // 16-byte pair (slots s, s + 1) holding columns cc, cc + 1 (cc even)
  __device__ static __forceinline__ void ld_pair(const float2* wave, int s, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(wave + s);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  }
  __device__ static __forceinline__ void st_pair(float2* wave, int s, float2 a, float2 b) {
    *reinterpret_cast<float4*>(wave + s) = make_float4(a.x, a.y, b.x, b.y);
  }
  // full barrier over the CTAs that share one wavefield
  __device__ static void sync_cluster() {
    if constexpr (G > 1) {
      cluster_arrive_release();
      cluster_wait();
    } else {
      __syncthreads();
    }
  }

  __device__ static __forceinline__ int rslot(int rank, int b, int r, int cc) { return slot<false>(rank, b, r, cc); }
  __device__ static __forceinline__ int cslot(int rank, int b, int r, int cc) { return slot<true>(rank, b, r, cc); }

  // Twiddles W_N^(n2 k1) = exp(-2 pi i n2 k1 / N): twS[k1*R2 + n2] (strided
  // stage, lanes over n2) and twC[n2*R1 + k1] (contiguous stage, lanes over
  // k1); fsq[p] = freq(nat(p))^2 for the band limit.
  __device__ static uint32_t bar_addr(const float2* wave, int which) {
    return smem_u32(wave) + (uint32_t)BAR_OFF + 8u * (uint32_t)which;
  }
  // Waits until every warp of this CTA has finished the stage and the
  // partner's block for this layout switch has arrived (bounded: gives up
  // after kExchangeSpin polls and flags it).  The mbarrier is the stage's
  // CTA barrier as well: each warp's arrival (after a warp barrier) releases
  // its lanes' writes and the completed phase acquires them, so no
  // __syncthreads is needed.
  __device__ static void exchange_wait(const float2* wave, int which, unsigned spin_limit = kExchangeSpin) {
    const uint32_t bar = bar_addr(wave, which);
    uint64_t tok = 0;
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tok = threadIdx.x == 0 ? mbar_arrive_tx(bar, BLK * 8) : mbar_arrive(bar);
    tok = __shfl_sync(0xffffffffu, tok, 0);
    unsigned it = 0;
    while (!mbar_try_wait(bar, tok)) {
      if (++it > spin_limit) {
        atomicOr(&g_exchange_timeouts, 1u);
        break;
      }
    }
  }

  // Layout switch of the 2-CTA tile: the stage writes its results in place
  // and every warp sends the off-diagonal slots it has just finished to the
  // same slots of the partner's idle buffer as bulk shared::cluster copies
  // that count their bytes on the partner's mbarrier `which`, so the
  // transfer overlaps the rest of the stage.  push() copies slots
  // [s0, s0 + n) of block `src` to block `dst` of the partner; the caller has
  // made the slots' writes visible to the copy engine (fence.proxy.async by
  // the writing threads, then a warp barrier).
  __device__ static void push(float2* wave, int rank, int src, int dst, int which, int s0, int n) {
    const uint32_t peer = (uint32_t)(rank ^ 1);
    const uint32_t from = smem_u32(wave + (size_t)src * BLK + s0);
    const uint32_t to = cluster_map(smem_u32(wave + (size_t)dst * BLK + s0), peer);
    const uint32_t bar = cluster_map(bar_addr(wave, which), peer);
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(to),
                 "r"(from), "r"((uint32_t)n * (uint32_t)sizeof(float2)), "r"(bar)
                 : "memory");
  }
  __device__ static void publish_warp() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
  }
  // Row -> column, after the row-contiguous round whose first task is that
  // of lane 0 (a): the warp's tasks (r, k1) of the off-diagonal block
  // b = rank ^ 1 cover whole 16-column groups, contiguous along each row.
  __device__ static void push_row_round(float2* wave, int rank, int a) {
    const int b = rank ^ 1;
    const int lane = threadIdx.x & 31;
    const int r = a / R1 + lane;  // one lane per row the warp touches
    if (lane < 32 / R1 + 2 && r < ROWS) {
      const int lo = max(a - R1 * r, NB * b), hi = min(a + 32 - R1 * r, NB * b + NB);
      if (lo < hi) push(wave, rank, 1, 2, 1, r * ROWS + R2 * (lo - NB * b), R2 * (hi - lo));
    }
  }
  // Column -> row, after the column-strided round whose first task is that
  // of lane 0 (a): one n2 and 32 consecutive columns, i.e. 32 contiguous
  // slots in each of the NB off-diagonal rows n2 + R2 j.
  __device__ static void push_col_round(float2* wave, int rank, int a) {
    const int lane = threadIdx.x & 31;
    if (lane < NB) {
      const int n2 = a / ROWS, cc0 = a % ROWS;
      push(wave, rank, 2, 1, 0, (n2 + R2 * lane) * ROWS + cc0, 32);
    }
  }

  __device__ static void init_tables(float2* twS, float2* twC, int* fsq) {
    if constexpr (XB) {
      if (threadIdx.x == 0) {
        const float2* wave = twS - WAVE;
        mbar_init(bar_addr(wave, 0), T / 32);
        mbar_init(bar_addr(wave, 1), T / 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
    }
    for (int i = threadIdx.x; i < N; i += T) {
      const int k1 = i / R2, n2 = i % R2;
      double s, c;
      sincospi(-2.0 * (double)(n2 * k1) / (double)N, &s, &c);
      twS[i] = make_float2((float)c, (float)s);
      const int n2b = i / R1, k1b = i % R1;
      sincospi(-2.0 * (double)(n2b * k1b) / (double)N, &s, &c);
      twC[i] = make_float2((float)c, (float)s);
      const int f = freq(nat(i));
      fsq[i] = f * f;
    }
  }

  // Row strided stage over the CTA's ROWS rows.  pre(grow, col) is called
  // first for every element of a task (global operands, issued before the
  // shared-memory work); FROM_SMEM: the values are the inverse s1' of the
  // slots (natural columns out), otherwise load(grow, col).  op(grow, col, v,
  // pre) sees natural real-space samples.  TO_SMEM: the forward s1 (R1-point
  // DFT + twiddle) is written back in place.  The caller synchronises.
  template <bool FROM_SMEM, bool TO_SMEM, class Load, class Pre, class Op>
  __device__ static void row_strided(float2* wave, const float2* twS, int rank, const Load& load, const Pre& pre,
                                     const Op& op) {
    // when T is a multiple of R2 every task of a thread has the same n2, so
    // its twiddles are loaded once per stage
    constexpr bool HOIST = TO_SMEM && (T % R2 == 0);
    float2 tw[R1];
    if constexpr (HOIST) {
#pragma unroll
      for (int k = 1; k < R1; ++k) tw[k] = twS[k * R2 + (int)(threadIdx.x % R2)];
    }
#pragma unroll 1
    for (int t = 0; t < SPT; ++t) {
      const int id = row_task<R2>(t);
      if (TS % T != 0 && id >= TS) break;
      const int r = id / R2, n2 = id % R2;
      const int grow = rank * ROWS + r;
      if (!chk(id >= 0 && grow < N && n2 + R2 * (R1 - 1) < N, kChkWindow)) continue;
      typename Pre::type pv[R1];
#pragma unroll
      for (int i = 0; i < R1; ++i) pv[i] = pre(grow, n2 + R2 * i);
      float2 x[R1];
      if constexpr (FROM_SMEM) {
#pragma unroll
        for (int i = 0; i < R1; ++i) {
          const int col = n2 + R2 * i;
          x[i] = wave[rslot(rank, col / ROWS, r, col % ROWS)];
        }
        Dft<R1, +1>::run(x);
      } else {
#pragma unroll
        for (int i = 0; i < R1; ++i) x[i] = load(grow, n2 + R2 * i);
      }
#pragma unroll
      for (int i = 0; i < R1; ++i) op(grow, n2 + R2 * i, x[i], pv[i]);
      if constexpr (TO_SMEM) {
        Dft<R1, -1>::run(x);
#pragma unroll
        for (int k = 1; k < R1; ++k) {
          if constexpr (HOIST) x[k] = cmul(x[k], tw[k]);
          else x[k] = cmul(x[k], twS[k * R2 + n2]);
        }
#pragma unroll
        for (int i = 0; i < R1; ++i) {
          const int col = n2 + R2 * i;
          wave[rslot(rank, col / ROWS, r, col % ROWS)] = x[i];
        }
      }
    }
  }

  // Row contiguous stage.  DIR < 0: forward s2, result to the column layout
  // (cluster block transpose when G > 1).  DIR > 0: inverse s2' + twiddle, in
  // place.  Ends with the barrier its result needs.
  template <int DIR>
  __device__ static void row_contig(float2* wave, const float2* twC, int rank) {
    if constexpr (DIR < 0 && G > 1 && !XB) {
      float2 x[CPT][R2];
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        const int id = row_task<R1>(t);
        if (TC % T != 0 && id >= TC) continue;
        const int r = id / R1, k1 = id % R1;
        const int b = k1 / NB, cc0 = R2 * (k1 % NB);
#pragma unroll
        for (int m = 0; m < R2; m += 2) ld_pair(wave, rslot(rank, b, r, cc0 + m), x[t][m], x[t][m + 1]);
      }
      // the DFTs consume every loaded value, so the loads have completed
      // before this thread arrives: the partner may then overwrite them
#pragma unroll
      for (int t = 0; t < CPT; ++t) Dft<R2, -1>::run(x[t]);
      cluster_arrive_relaxed();
      cluster_wait();
      const uint32_t w0 = smem_u32(wave);
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        const int id = row_task<R1>(t);
        if (TC % T != 0 && id >= TC) continue;
        const int r = id / R1, k1 = id % R1;
        const int b = k1 / NB, cc0 = R2 * (k1 % NB);
        if (b == rank) {
#pragma unroll
          for (int m = 0; m < R2; m += 2) st_pair(wave, cslot(rank, rank, r, cc0 + m), x[t][m], x[t][m + 1]);
        } else {
          const uint32_t base = cluster_map(w0, (uint32_t)b);
#pragma unroll
          for (int m = 0; m < R2; m += 2)
            st_cluster2(base + 8u * (uint32_t)cslot(b, rank, r, cc0 + m), x[t][m], x[t][m + 1]);
        }
      }
      cluster_arrive_release();
      cluster_wait();
    } else {
      // when T is a multiple of R1 every task of a thread has the same k1, so
      // the inverse stage's twiddles are loaded once per stage
      constexpr bool HOIST = DIR > 0 && (T % R1 == 0);
      float2 tw[R2];
      if constexpr (HOIST) {
#pragma unroll
        for (int i = 1; i < R2; ++i) tw[i] = twC[i * R1 + (int)(threadIdx.x % R1)];
      }
#pragma unroll 1
      for (int t = 0; t < CPT; ++t) {
        const int id = row_task<R1>(t);
        if (TC % T != 0 && id >= TC) break;
        const int r = id / R1, k1 = id % R1;
        const int b = k1 / NB, cc0 = R2 * (k1 % NB);
        float2 x[R2];
#pragma unroll
        for (int m = 0; m < R2; m += 2) ld_pair(wave, rslot(rank, b, r, cc0 + m), x[m], x[m + 1]);
        Dft<R2, DIR>::run(x);
        if constexpr (DIR > 0) {
#pragma unroll
          for (int i = 1; i < R2; ++i) {
            if constexpr (HOIST) x[i] = cmulc(x[i], tw[i]);
            else x[i] = cmulc(x[i], twC[i * R1 + k1]);
          }
        }
        // in place: the diagonal block has the same slots in both layouts,
        // the off-diagonal one goes to the partner's column-layout buffer
#pragma unroll
        for (int m = 0; m < R2; m += 2) st_pair(wave, rslot(rank, b, r, cc0 + m), x[m], x[m + 1]);
        if constexpr (DIR < 0 && XB) {
          publish_warp();
          push_row_round(wave, rank, id - (int)(threadIdx.x & 31));  // the warp's first task
        }
      }
      if constexpr (DIR < 0 && G > 1) {
        exchange_wait(wave, 1);
      } else if constexpr (DIR > 0) {
        row_sync();  // the next stage (real-space row stage) stays within rows
      } else {
        __syncthreads();
      }
    }
  }

  // Column strided stage.  DIR < 0: forward s1 (DFT + twiddle) in place.
  // DIR > 0: inverse s1', natural rows, result to the row layout (cluster
  // block transpose when G > 1).  Ends with the barrier its result needs.
  template <int DIR>
  __device__ static void col_strided(float2* wave, const float2* twS, int rank) {
    if constexpr (DIR > 0 && G > 1 && !XB) {
      float2 x[SPT][R1];
#pragma unroll
      for (int t = 0; t < SPT; ++t) {
        const int id = threadIdx.x + t * T;
        if (TS % T != 0 && id >= TS) continue;
        const int n2 = id / ROWS, cc = id % ROWS;
#pragma unroll
        for (int i = 0; i < R1; ++i) x[t][i] = wave[cslot(rank, i / NB, n2 + R2 * (i % NB), cc)];
      }
#pragma unroll
      for (int t = 0; t < SPT; ++t) Dft<R1, +1>::run(x[t]);
      cluster_arrive_relaxed();
      cluster_wait();
      const uint32_t w0 = smem_u32(wave);
      uint32_t base[G];
#pragma unroll
      for (int b = 0; b < G; ++b) base[b] = cluster_map(w0, (uint32_t)b);
#pragma unroll
      for (int t = 0; t < SPT; ++t) {
        const int id = threadIdx.x + t * T;
        if (TS % T != 0 && id >= TS) continue;
        const int n2 = id / ROWS, cc = id % ROWS;
#pragma unroll
        for (int i = 0; i < R1; ++i) {
          const int b = i / NB, r = n2 + R2 * (i % NB);
          if (b == rank) wave[rslot(rank, rank, r, cc)] = x[t][i];
          else st_cluster(base[b] + 8u * (uint32_t)rslot(b, rank, r, cc), x[t][i]);
        }
      }
      cluster_arrive_release();
      cluster_wait();
    } else {
#pragma unroll 1
      for (int t = 0; t < SPT; ++t) {
        const int id = threadIdx.x + t * T;
        if (TS % T != 0 && id >= TS) break;
        const int n2 = id / ROWS, cc = id % ROWS;
        float2 x[R1];
#pragma unroll
        for (int i = 0; i < R1; ++i) x[i] = wave[cslot(rank, i / NB, n2 + R2 * (i % NB), cc)];
        if constexpr (DIR < 0) {
          Dft<R1, -1>::run(x);
#pragma unroll
          for (int k = 1; k < R1; ++k) x[k] = cmul(x[k], twS[k * R2 + n2]);
#pragma unroll
          for (int i = 0; i < R1; ++i) wave[cslot(rank, i / NB, n2 + R2 * (i % NB), cc)] = x[i];
        } else {
          Dft<R1, +1>::run(x);
          // in place (the diagonal block has the same slots in both layouts;
          // the off-diagonal one goes to the partner's row-layout buffer)
#pragma unroll
          for (int i = 0; i < R1; ++i) wave[cslot(rank, i / NB, n2 + R2 * (i % NB), cc)] = x[i];
          if constexpr (XB) {
            publish_warp();
            push_col_round(wave, rank, (int)(threadIdx.x & ~31u) + t * T);
          }
        }
      }
      if constexpr (DIR > 0 && G > 1) {
        exchange_wait(wave, 0);
      } else {
        __syncthreads();
      }
    }
  }

  // Column contiguous stage on the spectral side.  Values come from the slots
  // (FROM_SMEM) or load(pu, pv); FWD applies the forward s2 so that register
  // i holds spectral slot pu = R2 k1 + i; op(pu, pv, v) is the pointwise
  // product; INV applies inverse s2' + twiddle and writes back in place; WB
  // (without INV) writes the spectral values back.  The caller synchronises.
  // With one warp per k1 (T = 32 R1) a thread keeps its k1 in every task
  // (columns lane + 32 t) and loads the inverse twiddles once per stage.
  static constexpr bool WARP_K1 = T == 32 * R1 && ROWS % 32 == 0;
  template <bool FROM_SMEM, bool FWD, bool INV, bool WB = false, class Load, class Op>
  __device__ static void col_contig(float2* wave, const float2* twC, int rank, const Load& load,
                                    const Op& op) {
    float2 tw[R2];
    if constexpr (INV && WARP_K1) {
#pragma unroll
      for (int i = 1; i < R2; ++i) tw[i] = twC[i * R1 + (int)(threadIdx.x / 32)];
    }
#pragma unroll 1
    for (int t = 0; t < CPT; ++t) {
      const int id = threadIdx.x + t * T;
      if (TC % T != 0 && id >= TC) break;
      const int k1 = WARP_K1 ? (int)(threadIdx.x / 32) : id / ROWS;
      const int cc = WARP_K1 ? (int)(threadIdx.x % 32) + 32 * t : id % ROWS;
      const int b = k1 / NB, r0 = R2 * (k1 % NB);
      const int pv = rank * ROWS + cc;
      const int pu0 = R2 * k1;
      if (!chk(pv >= 0 && pv < N && pu0 >= 0 && pu0 + R2 <= N, kChkWindow)) continue;
      float2 x[R2];
      if constexpr (FROM_SMEM) {
#pragma unroll
        for (int i = 0; i < R2; ++i) x[i] = wave[cslot(rank, b, r0 + i, cc)];
      } else {
#pragma unroll
        for (int i = 0; i < R2; ++i) x[i] = load(pu0 + i, pv);
      }
      if constexpr (FWD) Dft<R2, -1>::run(x);
#pragma unroll
      for (int i = 0; i < R2; ++i) op(pu0 + i, pv, x[i]);
      if constexpr (INV) {
        Dft<R2, +1>::run(x);
#pragma unroll
        for (int i = 1; i < R2; ++i) {
          if constexpr (WARP_K1) x[i] = cmulc(x[i], tw[i]);
          else x[i] = cmulc(x[i], twC[i * R1 + k1]);
        }
#pragma unroll
        for (int i = 0; i < R2; ++i) wave[cslot(rank, b, r0 + i, cc)] = x[i];
      } else if constexpr (WB) {
#pragma unroll
        for (int i = 0; i < R2; ++i) wave[cslot(rank, b, r0 + i, cc)] = x[i];
      }
    }
  }

  // ---- composite passes -------------------------------------------------
  // Inverse 2-D transform from a spectrum already in the column layout,
  // after its contiguous stage: column s1' (to row layout), row s2'.  The
  // row s1' is left to the caller (fused with the next pointwise op).
  __device__ static void inverse_tail(float2* wave, const float2* twS, const float2* twC, int rank) {
    col_strided<+1>(wave, twS, rank);
    row_contig<+1>(wave, twC, rank);
  }
  // Forward 2-D transform after the row s1 stage: row s2 (to column
  // layout), column s1.  The column s2 is left to the caller.
  __device__ static void forward_mid(float2* wave, const float2* twS, const float2* twC, int rank) {
    row_contig<-1>(wave, twC, rank);
    col_strided<-1>(wave, twS, rank);
  }
};

}  // namespace ptycho
