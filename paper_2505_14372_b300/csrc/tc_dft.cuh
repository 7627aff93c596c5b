// Small complex DFTs as tensor-core GEMMs (warp-level mma.sync), with the
// fp32 operands split into lower-precision terms whose largest cross
// products recover near-fp32 accuracy (precision variant of the FFT tile).
//
// One call transforms 8 tasks (vectors of R <= 16 complex values) at once:
//   Y = M X,  X: 32 x 8 (rows 0-15 real parts, 16-31 imaginary parts of the
//   task's elements, zero-padded beyond R), M: 32 x 32 = [[Wr, -Wi], [Wi, Wr]]
//   with W[m][e] = exp(DIR 2 pi i m e / R).
// Modes: TF32X3 (x = hi + lo in tf32, hi*hi + hi*lo + lo*hi on m16n8k8),
// BF16X3 (the same with bf16 on m16n8k16), TF32X1 (one tf32 product),
// BF16X6 (x = x0 + x1 + x2 in bf16, 8 significand bits each, so the three
// parts hold all 24 bits of an fp32 value; the six products x_i y_j with
// i + j <= 2, whose dropped terms are below 2^-24 relative).
// Fragment ownership (PTX m16n8k8 / m16n8k16 layouts), g = lane/4, t = lane%4:
//   TF32: lane loads elements {t, t+4, t+8, t+12} of task g;
//   BF16: lane loads elements {2t, 2t+1, 2t+8, 2t+9} of task g;
//   both: lane receives outputs m in {g, g+8} of tasks {2t, 2t+1}.
// The matrices' fragments are tables built on the host in FP64 and split
// there (tc_tables), indexed [lane][register] so that each lane's loads are
// contiguous.
// Accumulation in the split modes: the MMA adds its accumulator input to the
// products after aligning them to the largest and truncating, so every MMA
// whose input already holds the full-size result loses low bits of it.  The
// small cross products therefore run as one chain of their own (its sums
// stay 2^-8 or less of the result), while the leading product of each
// k-step starts from a zero accumulator and the k-steps' leading sums are
// added with round-to-nearest fp32 adds: two (bf16) or four (tf32)
// truncations at full size per output instead of one per MMA.
#pragma once
#include <stdint.h>

#include "radix.cuh"

namespace ptycho {

enum TcMode { TC_NONE = 0, TC_TF32X3 = 1, TC_BF16X3 = 2, TC_TF32X1 = 3, TC_BF16X6 = 4 };
constexpr int kTcModes = 4;

template <int MODE>
__host__ __device__ constexpr bool tc_is_bf16() { return MODE == TC_BF16X3 || MODE == TC_BF16X6; }
// operand parts of a split mode
template <int MODE>
__host__ __device__ constexpr int tc_parts() { return MODE == TC_BF16X6 ? 3 : MODE == TC_TF32X1 ? 1 : 2; }

// words per lane in a fragment table (the TF32x3 size; BF16x3 uses half)
constexpr int kTcLaneWords = 64;

// registers of A fragments per lane for one (R, DIR) matrix
template <int MODE>
struct TcRegs {
  // TF32: 2 m-tiles x 4 k-steps x 4 regs, hi and lo; BF16: 2 x 2 x 4 per
  // part (two parts, or three for BF16X6)
  static constexpr int N = MODE == TC_BF16X6 ? 48 : MODE == TC_BF16X3 ? 32 : 64;
};

__device__ __forceinline__ uint32_t f2tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
  // element with the lower row index in the low half
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_elem), "f"(lo_elem));
  return r;
}
__device__ __forceinline__ float bf16_lo_as_float(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi_as_float(uint32_t p) { return __uint_as_float(p & 0xffff0000u); }
// (v0, v1) as PARTS packed bf16 pairs, most significant first: each part is
// the rounded remainder of the ones before it (the remainders are exact in
// fp32)
template <int PARTS>
__device__ __forceinline__ void split_bf16(float v0, float v1, uint32_t (&p)[PARTS]) {
#pragma unroll
  for (int i = 0; i < PARTS; ++i) {
    p[i] = pack_bf16(v0, v1);
    v0 -= bf16_lo_as_float(p[i]);
    v1 -= bf16_hi_as_float(p[i]);
  }
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragments of one DFT matrix held by the calling lane.
template <int MODE>
struct TcMat {
  uint32_t a[TcRegs<MODE>::N];
  __device__ __forceinline__ void load(const uint32_t* table) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < TcRegs<MODE>::N; ++i) a[i] = __ldg(table + lane * kTcLaneWords + i);
  }
};

// Transforms tasks task0..task0+7.  ld(task, e) -> float2 input element e
// (only called for e < R); st(task, m, float2) receives output m < R.
// CONJ: the opposite direction from the same fragments.  The DFT matrix is
// symmetric, so the real form of the other direction, [[Wr, Wi], [-Wi, Wr]],
// is M with its off-diagonal blocks negated: the sign bits of every part of
// those fragments are flipped (rounding to tf32 / bf16 is symmetric, so the
// parts of -x are the negated parts of x).  One matrix per stage then
// serves both directions.
template <int MODE, int R, bool CONJ = false, class Ld, class St>
__device__ __forceinline__ void tc_dft8(const TcMat<MODE>& M, int task0, const Ld& ld, const St& st) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  // d: result (the one chain of TF32X1, else the small cross products);
  // e: the split modes' leading products, summed one k-step at a time
  float d[2][4], e[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int i = 0; i < 4; ++i) d[mt][i] = e[mt][i] = 0.f;
  // leading product of one k-step from a zero accumulator, added to e
  auto lead = [&](int mt, float(&t)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) e[mt][i] += t[i];
  };
  if constexpr (tc_is_bf16<MODE>()) {
    constexpr int NPART = tc_parts<MODE>();
    // elements 2t, 2t+1, 2t+8, 2t+9 of task g
    float2 x[4];
    const int es[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = es[j] < R ? ld(task0 + g, es[j]) : make_float2(0.f, 0.f);
    // k-step 0: real parts, k-step 1: imaginary parts; b[ks][r][part]
    uint32_t b[2][2][NPART];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      split_bf16<NPART>(ks ? x[0].y : x[0].x, ks ? x[1].y : x[1].x, b[ks][0]);
      split_bf16<NPART>(ks ? x[2].y : x[2].x, ks ? x[3].y : x[3].x, b[ks][1]);
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        // part q of the matrix fragment (sign bits of both bf16 halves
        // flipped in the off-diagonal blocks of the opposite direction)
        const uint32_t fl = (CONJ && mt != ks) ? 0x80008000u : 0u;
        auto A = [&](int q) {
          const uint32_t* a = &M.a[16 * q + (mt * 2 + ks) * 4];
          return a;
        };
        // the products a_i b_j with i + j <= NPART - 1, smallest first
        auto prod = [&](int i, int j) {
          const uint32_t* a = A(i);
          const uint32_t AF[4] = {a[0] ^ fl, a[1] ^ fl, a[2] ^ fl, a[3] ^ fl};
          mma_bf16(d[mt], AF, b[ks][0][j], b[ks][1][j]);
        };
        if constexpr (NPART == 3) {
          prod(0, 2);
          prod(1, 1);
          prod(2, 0);
        }
        prod(1, 0);
        prod(0, 1);
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t* a = A(0);
        const uint32_t AF[4] = {a[0] ^ fl, a[1] ^ fl, a[2] ^ fl, a[3] ^ fl};
        mma_bf16(t, AF, b[ks][0][0], b[ks][1][0]);
        lead(mt, t);
      }
  } else {
    // elements t, t+4, t+8, t+12 of task g
    float2 x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = (t + 4 * j) < R ? ld(task0 + g, t + 4 * j) : make_float2(0.f, 0.f);
    // k-steps: 0 re(t, t+4), 1 re(t+8, t+12), 2 im(t, t+4), 3 im(t+8, t+12)
    float v[4][2] = {{x[0].x, x[1].x}, {x[2].x, x[3].x}, {x[0].y, x[1].y}, {x[2].y, x[3].y}};
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        // k-steps 2, 3 read imaginary parts: off-diagonal when mt == 0
        const uint32_t fl = (CONJ && mt != (kk >= 2 ? 1 : 0)) ? 0x80000000u : 0u;
        const uint32_t* ah = &M.a[(mt * 4 + kk) * 4];
        const uint32_t AH[4] = {ah[0] ^ fl, ah[1] ^ fl, ah[2] ^ fl, ah[3] ^ fl};
        const uint32_t b0h = f2tf32(v[kk][0]), b1h = f2tf32(v[kk][1]);
        if constexpr (MODE == TC_TF32X3) {
          const uint32_t* al = &M.a[32 + (mt * 4 + kk) * 4];
          const uint32_t AL[4] = {al[0] ^ fl, al[1] ^ fl, al[2] ^ fl, al[3] ^ fl};
          const uint32_t b0l = f2tf32(v[kk][0] - __uint_as_float(b0h));
          const uint32_t b1l = f2tf32(v[kk][1] - __uint_as_float(b1h));
          mma_tf32(d[mt], AL, b0h, b1h);
          mma_tf32(d[mt], AH, b0l, b1l);
          float t[4] = {0.f, 0.f, 0.f, 0.f};
          mma_tf32(t, AH, b0h, b1h);
          lead(mt, t);
        } else {
          mma_tf32(d[mt], AH, b0h, b1h);
        }
      }
  }
  if constexpr (MODE != TC_TF32X1) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) d[mt][i] = e[mt][i] + d[mt][i];
  }
  // outputs: rows g and g+8 (real in m-tile 0, imaginary in m-tile 1), tasks 2t and 2t+1
  if (g < R) {
    st(task0 + 2 * t, g, make_float2(d[0][0], d[1][0]));
    st(task0 + 2 * t + 1, g, make_float2(d[0][1], d[1][1]));
  }
  if (g + 8 < R) {
    st(task0 + 2 * t, g + 8, make_float2(d[0][2], d[1][2]));
    st(task0 + 2 * t + 1, g + 8, make_float2(d[0][3], d[1][3]));
  }
}

}  // namespace ptycho
