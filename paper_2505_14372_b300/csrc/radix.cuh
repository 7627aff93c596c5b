// Register-level complex arithmetic and small DFTs for the shared-memory
// FFT tile (sm_103a).  All values are interleaved complex64 (float2).
//
// Sign convention: DIR = -1 is the forward kernel exp(-2 pi i k n / R),
// DIR = +1 the inverse kernel exp(+2 pi i k n / R) (unnormalised).
#pragma once
#include <cuda_runtime.h>

namespace ptycho {

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// multiply by -i (DIR < 0) or +i (DIR > 0)
template <int DIR>
__host__ __device__ __forceinline__ float2 rot90(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}


// cos and sin of 2*pi*m/48 (m = 0..47): every twiddle of the 8-, 12- and
// 16-point register DFTs is one of these angles (multiples of 7.5 degrees);
// the values are the exact trigonometric constants rounded to float.
__host__ __host__ __device__ __forceinline__ constexpr float cos48(int m) {
  switch (((m % 48) + 48) % 48) {
    case 0: return 1.0f;
    case 1: return 0.99144486137381038f;
    case 2: return 0.96592582628906831f;
    case 3: return 0.92387953251128674f;
    case 4: return 0.86602540378443871f;
    case 5: return 0.79335334029123517f;
    case 6: return 0.70710678118654757f;
    case 7: return 0.60876142900872066f;
    case 8: return 0.5f;
    case 9: return 0.38268343236508984f;
    case 10: return 0.25881904510252074f;
    case 11: return 0.13052619222005171f;
    case 12: return 0.0f;
    case 13: return -0.1305261922200516f;
    case 14: return -0.25881904510252063f;
    case 15: return -0.3826834323650895f;
    case 16: return -0.5f;
    case 17: return -0.60876142900872066f;
    case 18: return -0.70710678118654746f;
    case 19: return -0.79335334029123505f;
    case 20: return -0.86602540378443871f;
    case 21: return -0.92387953251128674f;
    case 22: return -0.9659258262890682f;
    case 23: return -0.99144486137381038f;
    case 24: return -1.0f;
    case 25: return -0.99144486137381038f;
    case 26: return -0.96592582628906831f;
    case 27: return -0.92387953251128685f;
    case 28: return -0.86602540378443882f;
    case 29: return -0.79335334029123517f;
    case 30: return -0.70710678118654791f;
    case 31: return -0.60876142900872088f;
    case 32: return -0.5f;
    case 33: return -0.3826834323650895f;
    case 34: return -0.25881904510252063f;
    case 35: return -0.13052619222005163f;
    case 36: return 0.0f;
    case 37: return 0.13052619222005127f;
    case 38: return 0.2588190451025203f;
    case 39: return 0.38268343236508917f;
    case 40: return 0.5f;
    case 41: return 0.60876142900871988f;
    case 42: return 0.70710678118654735f;
    case 43: return 0.79335334029123494f;
    case 44: return 0.86602540378443837f;
    case 45: return 0.92387953251128685f;
    case 46: return 0.96592582628906809f;
    case 47: return 0.99144486137381038f;
  }
  return 0.0f;
}
__host__ __host__ __device__ __forceinline__ constexpr float sin48(int m) {
  switch (((m % 48) + 48) % 48) {
    case 0: return 0.0f;
    case 1: return 0.13052619222005157f;
    case 2: return 0.25881904510252074f;
    case 3: return 0.38268343236508978f;
    case 4: return 0.5f;
    case 5: return 0.60876142900872066f;
    case 6: return 0.70710678118654746f;
    case 7: return 0.79335334029123517f;
    case 8: return 0.8660254037844386f;
    case 9: return 0.92387953251128674f;
    case 10: return 0.96592582628906831f;
    case 11: return 0.99144486137381038f;
    case 12: return 1.0f;
    case 13: return 0.99144486137381038f;
    case 14: return 0.96592582628906831f;
    case 15: return 0.92387953251128685f;
    case 16: return 0.86602540378443871f;
    case 17: return 0.79335334029123517f;
    case 18: return 0.70710678118654757f;
    case 19: return 0.60876142900872088f;
    case 20: return 0.5f;
    case 21: return 0.38268343236508989f;
    case 22: return 0.25881904510252102f;
    case 23: return 0.13052619222005199f;
    case 24: return 0.0f;
    case 25: return -0.13052619222005177f;
    case 26: return -0.25881904510252079f;
    case 27: return -0.38268343236508967f;
    case 28: return -0.5f;
    case 29: return -0.60876142900872066f;
    case 30: return -0.70710678118654713f;
    case 31: return -0.79335334029123494f;
    case 32: return -0.86602540378443837f;
    case 33: return -0.92387953251128685f;
    case 34: return -0.96592582628906831f;
    case 35: return -0.99144486137381038f;
    case 36: return -1.0f;
    case 37: return -0.99144486137381049f;
    case 38: return -0.96592582628906842f;
    case 39: return -0.92387953251128696f;
    case 40: return -0.8660254037844386f;
    case 41: return -0.79335334029123572f;
    case 42: return -0.70710678118654768f;
    case 43: return -0.60876142900872088f;
    case 44: return -0.5f;
    case 45: return -0.38268343236508956f;
    case 46: return -0.25881904510252157f;
    case 47: return -0.13052619222005168f;
  }
  return 0.0f;
}

// v * exp(DIR * 2 pi i * m / R) for a compile-time-foldable m (R divides 48).
template <int R, int DIR>
__host__ __device__ __forceinline__ float2 twiddle(float2 v, int m) {
  static_assert(48 % R == 0, "radix must divide 48");
  const int a = ((m * (48 / R)) % 48 + 48) % 48;
  if (a == 0) return v;
  if (a == 12) return rot90<DIR>(v);   // exp(DIR i pi/2) = DIR i
  if (a == 24) return make_float2(-v.x, -v.y);
  if (a == 36) return rot90<-DIR>(v);  // exp(DIR i 3pi/2) = -DIR i
  const float c = cos48(a);
  const float s = DIR < 0 ? -sin48(a) : sin48(a);
  return cmul(v, make_float2(c, s));
}

template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<1, DIR> {
  __host__ __device__ __forceinline__ static void run(float2*) {}
};

template <int DIR> struct Dft<2, DIR> {
  __host__ __device__ __forceinline__ static void run(float2* x) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

// 3-point: X1,2 = x0 - (x1+x2)/2 -+ DIR-rotated (sqrt(3)/2)(x1-x2)
template <int DIR> struct Dft<3, DIR> {
  __host__ __device__ __forceinline__ static void run(float2* x) {
    const float2 t1 = cadd(x[1], x[2]);
    const float2 t2 = csub(x[1], x[2]);
    const float2 m = make_float2(fmaf(-0.5f, t1.x, x[0].x), fmaf(-0.5f, t1.y, x[0].y));
    const float2 r = cscale(rot90<DIR>(t2), 0.86602540378443865f);
    x[0] = cadd(x[0], t1);
    x[1] = cadd(m, r);
    x[2] = csub(m, r);
  }
};

template <int DIR> struct Dft<4, DIR> {
  __host__ __device__ __forceinline__ static void run(float2* x) {
    const float2 a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
    const float2 c = cadd(x[1], x[3]), d = rot90<DIR>(csub(x[1], x[3]));
    x[0] = cadd(a, c);
    x[2] = csub(a, c);
    x[1] = cadd(b, d);
    x[3] = csub(b, d);
  }
};

// R = A*B by one Cooley-Tukey split: input index n = b + B a, output
// k = ka + A kb; inner A-point DFTs, twiddles W_R^(b ka), outer B-point DFTs.
template <int A, int B, int DIR>
__host__ __device__ __forceinline__ void dft_split(float2* x) {
  constexpr int R = A * B;
  float2 y[B][A];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    float2 t[A];
#pragma unroll
    for (int a = 0; a < A; ++a) t[a] = x[b + B * a];
    Dft<A, DIR>::run(t);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) y[b][ka] = twiddle<R, DIR>(t[ka], b * ka);
  }
#pragma unroll
  for (int ka = 0; ka < A; ++ka) {
    float2 t[B];
#pragma unroll
    for (int b = 0; b < B; ++b) t[b] = y[b][ka];
    Dft<B, DIR>::run(t);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) x[ka + A * kb] = t[kb];
  }
}

template <int DIR> struct Dft<8, DIR> {
  __host__ __device__ __forceinline__ static void run(float2* x) { dft_split<4, 2, DIR>(x); }
};
template <int DIR> struct Dft<12, DIR> {
  __host__ __device__ __forceinline__ static void run(float2* x) { dft_split<4, 3, DIR>(x); }
};
template <int DIR> struct Dft<16, DIR> {
  __host__ __device__ __forceinline__ static void run(float2* x) { dft_split<4, 4, DIR>(x); }
};

}  // namespace ptycho
