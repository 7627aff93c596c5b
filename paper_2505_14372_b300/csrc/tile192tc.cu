// Tensor-core DFT variant of the 192x192 tile (2-CTA cluster): TF32x3,
// BF16x3, TF32x1 and BF16x6 modes.  Also builds the DFT-matrix fragment tables.
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "ctxid.h"
#include "engine_impl.cuh"
#include "ptycho.h"
#include "tile_tc.cuh"

namespace ptycho {

namespace {

uint32_t f32_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
}
float bits_f32(uint32_t u) {
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}
// round to tf32 (10 mantissa bits), nearest, ties away from zero
float to_tf32(float x) {
  uint32_t u = f32_bits(x);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  return bits_f32(u);
}
// round to bf16, nearest even
uint16_t to_bf16(float x) {
  const uint32_t u = f32_bits(x);
  const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(r >> 16);
}
float bf16_to_f32(uint16_t b) { return bits_f32((uint32_t)b << 16); }

// Real 32 x 32 matrix of the complex R-point DFT (rows: real then imaginary
// outputs, columns: real then imaginary inputs), zero beyond R.
double dft_real(int R, int dir, int row, int col) {
  const int m = row % 16, e = col % 16;
  if (m >= R || e >= R) return 0.0;
  const double a = 2.0 * M_PI * (double)((m * e) % R) / (double)R;
  const double wr = std::cos(a), wi = dir * std::sin(a);
  const bool out_im = row >= 16, in_im = col >= 16;
  if (!out_im && !in_im) return wr;
  if (!out_im && in_im) return -wi;
  if (out_im && !in_im) return wi;
  return wr;
}

void fill_table(int mode, int R, int dir, uint32_t* out) {
  for (int lane = 0; lane < 32; ++lane) {
    const int g = lane / 4, t = lane % 4;
    uint32_t* o = out + lane * kTcLaneWords;
    if (mode == TC_BF16X3 || mode == TC_BF16X6) {
      // m16n8k16 A fragment: {A[g][2t], A[g][2t+1]}, {A[g+8][..]}, {A[g][2t+8], ..}, {A[g+8][2t+8], ..};
      // part q (the rounded remainder of the parts before it) at word 16 q
      const int parts = mode == TC_BF16X6 ? 3 : 2;
      for (int mt = 0; mt < 2; ++mt)
        for (int ks = 0; ks < 2; ++ks)
          for (int reg = 0; reg < 4; ++reg) {
            const int row = 16 * mt + g + ((reg & 1) ? 8 : 0);
            const int col = 16 * ks + 2 * t + ((reg & 2) ? 8 : 0);
            uint32_t w[3] = {0, 0, 0};
            for (int h = 0; h < 2; ++h) {
              double v = dft_real(R, dir, row, col + h);
              for (int q = 0; q < parts; ++q) {
                const uint16_t b = to_bf16((float)v);
                v -= (double)bf16_to_f32(b);
                w[q] |= (uint32_t)b << (16 * h);
              }
            }
            for (int q = 0; q < parts; ++q) o[16 * q + (mt * 2 + ks) * 4 + reg] = w[q];
          }
    } else {
      // m16n8k8 A fragment: A[g][t], A[g+8][t], A[g][t+4], A[g+8][t+4]
      for (int mt = 0; mt < 2; ++mt)
        for (int kk = 0; kk < 4; ++kk)
          for (int reg = 0; reg < 4; ++reg) {
            const int row = 16 * mt + g + ((reg & 1) ? 8 : 0);
            const int col = 8 * kk + t + ((reg & 2) ? 4 : 0);
            const double v = dft_real(R, dir, row, col);
            const float h = to_tf32((float)v);
            const float l = to_tf32((float)(v - (double)h));
            o[(mt * 4 + kk) * 4 + reg] = f32_bits(h);
            o[32 + (mt * 4 + kk) * 4 + reg] = f32_bits(l);
          }
    }
  }
}

std::mutex g_mu;
std::set<unsigned long long> g_ready;  // contexts whose tables are filled

// Fills the fragment tables once per CUDA context (a __device__ array
// exists once per context).
cudaError_t ensure_tables(int R1, int R2) {
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = 0;
  if (ptycho::current_context_id(&id) != PTYCHO_OK) return cudaErrorUnknown;
  if (id != 0 && g_ready.count(id)) return cudaSuccess;
  std::vector<uint32_t> h((size_t)kTcModes * 4 * kTcTableWords, 0u);
  const int modes[kTcModes] = {TC_TF32X3, TC_BF16X3, TC_TF32X1, TC_BF16X6};
  for (int mi = 0; mi < kTcModes; ++mi)
    for (int m = 0; m < 4; ++m)
      fill_table(modes[mi], m < 2 ? R1 : R2, (m & 1) ? +1 : -1, &h[((size_t)mi * 4 + m) * kTcTableWords]);
  const cudaError_t e = cudaMemcpyToSymbol(g_tc_tables, h.data(), h.size() * 4);
  // the copy binds the primary context when none was current
  if (e == cudaSuccess && (id != 0 || ptycho::current_context_id(&id) == PTYCHO_OK) && id != 0) g_ready.insert(id);
  return e;
}

template <int MODE>
struct TcEngine {
  using TL = TileTC<Tile<192, 2, 16, 384, 1>, MODE>;
  using E = Engine<TL, false>;  // FP32 entry waves and the gradient only
  static cudaError_t probe_spectrum(const float2* P, float2* Phat, int K, cudaStream_t s) {
    cudaError_t e = ensure_tables(TL::R1, TL::R2);
    return e != cudaSuccess ? e : E::probe_spectrum(P, Phat, K, s);
  }
  static cudaError_t forward(const LaunchArgs& L, int clusters, bool store, int variant, cudaStream_t s) {
    cudaError_t e = ensure_tables(TL::R1, TL::R2);
    return e != cudaSuccess ? e : E::forward(L, clusters, store, variant, s);
  }
  static cudaError_t adjoint(const LaunchArgs& L, int clusters, bool store, int variant, cudaStream_t s) {
    cudaError_t e = ensure_tables(TL::R1, TL::R2);
    return e != cudaSuccess ? e : E::adjoint(L, clusters, store, variant, s);
  }
  static cudaError_t adjoint_pos(const LaunchArgs& L, const PosArgs& F, int clusters, int variant, cudaStream_t s) {
    cudaError_t e = ensure_tables(TL::R1, TL::R2);
    return e != cudaSuccess ? e : E::adjoint_pos(L, F, clusters, variant, s);
  }
  static cudaError_t probe_grad(const float2* gPhat, float2* gP, int K, int acc, cudaStream_t s) {
    cudaError_t e = ensure_tables(TL::R1, TL::R2);
    return e != cudaSuccess ? e : E::probe_grad(gPhat, gP, K, acc, s);
  }
  static cudaError_t fft_debug(const float2* in, float2* out, int count, int dir, cudaStream_t s) {
    cudaError_t e = ensure_tables(TL::R1, TL::R2);
    return e != cudaSuccess ? e : E::fft_debug(in, out, count, dir, s);
  }
  static const EngineOps* ops() {
    static const EngineOps o = [] {
      EngineOps x = *E::ops();
      x.probe_spectrum = &probe_spectrum;
      x.forward = &forward;
      x.adjoint = &adjoint;
      x.probe_grad = &probe_grad;
      x.adjoint_pos = &adjoint_pos;
      x.fft_debug = &fft_debug;
      return x;
    }();
    return &o;
  }
};

}  // namespace

const EngineOps* engine_192_tc(int mode) {
  switch (mode) {
    case TC_TF32X3: return TcEngine<TC_TF32X3>::ops();
    case TC_BF16X3: return TcEngine<TC_BF16X3>::ops();
    case TC_TF32X1: return TcEngine<TC_TF32X1>::ops();
    case TC_BF16X6: return TcEngine<TC_BF16X6>::ops();
    default: return nullptr;
  }
}

}  // namespace ptycho
