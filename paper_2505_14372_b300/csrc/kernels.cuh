// Kernels of the batched mixed-state multislice forward model and its
// adjoint (arXiv 2505.14372 §3, §3.1, §3.2), one template per tile shape.
//
// A work item is one (scan position j, probe mode k) pair of one problem
// descriptor; a cluster of G CTAs owns one item at a time and keeps its
// wavefield in shared memory across all slices.  Items of several problems
// with the same window size may share one launch (serving).
#pragma once
#include <float.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "elementwise.cuh"
#include "launch.h"
#include "noise.cuh"
#include "tile.cuh"

namespace ptycho {

// Entry-wave copies between the forward pass and the object-gradient term:
// FP32, binary16 or bfloat16 per part (PREC 0 / 1 / 2), rounded to nearest
// even on the way out, widened exactly on the way back.  The format is a
// template parameter of the kernels, so the prefetched loads stay
// branch-free.
template <int PREC>
__device__ __forceinline__ void wave_put(char* base, int i, float2 v) {
  // streaming stores: the entry waves are read back once, after every mode's
  // forward pass, so they should not displace the object patch in L2
  if constexpr (PREC == 0) {
    __stcs(reinterpret_cast<float2*>(base) + i, v);
  } else {
    unsigned u;
    if constexpr (PREC == 1) {
      const __half2 h = __floats2half2_rn(v.x, v.y);
      memcpy(&u, &h, sizeof(u));
    } else {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
      memcpy(&u, &h, sizeof(u));
    }
    __stcs(reinterpret_cast<unsigned*>(base) + i, u);
  }
}
template <int PREC>
__device__ __forceinline__ float2 wave_get(const char* base, int i) {
  if constexpr (PREC == 0) {
    return __ldcs(reinterpret_cast<const float2*>(base) + i);
  } else {
    const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(base) + i);
    if constexpr (PREC == 1) {
      __half2 h;
      memcpy(&h, &u, sizeof(u));
      return __half22float2(h);
    } else {
      // bfloat16: the high half of a binary32 (real part in the low 16 bits)
      return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
  }
}
// Compile-time properties of a kernel variant (launch.h: Variant).
template <int V>
struct Var {
  static constexpr int prec = V <= kVarBF16 ? V : 0;  // entry-wave storage format
  static constexpr bool epie = V == kVarEpie;         // ePIE normalisers (§3.3.1)
  static constexpr bool lsq_dir = V == kVarLsqDir;    // LSQML direction pass (§3.3.2)
  static constexpr bool lsq_step = V == kVarLsqStep;  // LSQML step-size pass
  static constexpr bool det = V == kVarDet;           // per-position gradients, fixed-order sums later
  static constexpr size_t wave_bytes = prec ? 4 : 8;
  // entry waves per mode in a slot: S, plus the shifted probe direction in
  // the step pass
  static constexpr int extra_waves = lsq_step ? 1 : 0;
};

// Programmatic dependent launch: kernels launched with programmatic stream
// serialization may start while the kernel before them in the stream is
// finishing; each waits (griddepcontrol.wait: the prerequisite grid has
// completed and its memory is visible) after its own set-up and before it
// reads anything an earlier kernel wrote, and lets the next kernel start
// once its main work is issued.  Both are no-ops in a launch without the
// attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void red_add1(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ const ProblemDesc& find_desc(const LaunchArgs& L, int item) {
  int d = 0;
#pragma unroll 1
  while (d + 1 < L.nd && item >= L.d[d + 1].item0) ++d;
  return L.d[d];
}

// Patch origin n = floor(r + 1/2) and subpixel part r - n (FP64).
struct ItemGeo {
  int j, jj, k, ny, nx;
  double dy, dx;
  bool ok;
};

template <class TL>
__device__ __forceinline__ ItemGeo item_geo(const ProblemDesc& D, int item) {
  ItemGeo g;
  const int local = item - D.item0;
  g.j = local / D.K;
  g.k = local - g.j * D.K;
  if (!chk(local >= 0 && g.j < D.B, kChkItem)) {  // checked build: an item outside its problem
    g.j = g.k = g.jj = 0;
    g.ok = false;
    g.ny = g.nx = 0;
    g.dy = g.dx = 0.0;
    return g;
  }
  g.jj = D.idx ? D.idx[g.j] : g.j;
  if (g.jj < 0 || g.jj >= D.npos) {
    g.ok = false;
    g.ny = g.nx = 0;
    g.dy = g.dx = 0.0;
    return g;
  }
  const double ry = (double)D.pos[2 * (size_t)g.jj], rx = (double)D.pos[2 * (size_t)g.jj + 1];
  const double fy = floor(ry + 0.5), fx = floor(rx + 0.5);
  g.dy = ry - fy;
  g.dx = rx - fx;
  g.ok = fy >= 0.0 && fx >= 0.0 && fy + TL::N <= (double)D.H && fx + TL::N <= (double)D.W;
  g.ny = g.ok ? (int)fy : 0;
  g.nx = g.ok ? (int)fx : 0;
  return g;
}

// Separable Fourier phase ramp exp(-2 pi i f delta / N) per spectral slot;
// the phase is formed in turns in FP64 and reduced to [-1/2, 1/2] first.
template <class TL>
__device__ __forceinline__ void make_ramps(float2* rampY, float2* rampX, double dy, double dx) {
  for (int p = threadIdx.x; p < TL::N; p += TL::T) {
    const double f = (double)TL::freq(TL::nat(p));
    double ty = f * dy / (double)TL::N, tx = f * dx / (double)TL::N;
    ty -= rint(ty);
    tx -= rint(tx);
    float s, c;
    sincospif(-2.0f * (float)ty, &s, &c);
    rampY[p] = make_float2(c, s);
    sincospif(-2.0f * (float)tx, &s, &c);
    rampX[p] = make_float2(c, s);
  }
}

template <class TL>
struct Smem {
  float2* wave;
  float2* twS;
  float2* twC;
  float2* rampY;
  float2* rampX;
  float2* chirp;  // [2][N]
  int* fsq;
  __device__ Smem(float4* raw) {
    wave = reinterpret_cast<float2*>(raw);
    twS = wave + TL::WAVE;
    twC = twS + TL::N;
    rampY = twC + TL::N;
    rampX = rampY + TL::N;
    chirp = rampX + TL::N;
    fsq = reinterpret_cast<int*>(chirp + 2 * TL::N);
  }
};

// Global operands of the real-space stage, issued before its shared-memory
// work so that their latency overlaps the inverse DFT.
struct PreO {
  const float2* O;
  int W;
  using type = float2;
  __device__ float2 operator()(int r, int c) const { return __ldg(O + (size_t)r * W + c); }
};
struct PsiO {
  float2 psi, o;
};
template <int PREC>
struct PrePsiO {
  const char* psi;  // entry wave of the slice, natural order, row stride N, format PREC
  int N;
  const float2* O;
  int W;
  using type = PsiO;
  __device__ PsiO operator()(int r, int c) const {
    return {wave_get<PREC>(psi, r * N + c), __ldg(O + (size_t)r * W + c)};
  }
};

template <class TL>
__device__ __forceinline__ void load_chirp(float2* dst, const float2* src) {
  for (int p = threadIdx.x; p < TL::N; p += TL::T) dst[p] = src[p];
}

// Propagator product on the spectral side: H(pu,pv) = h[pu] h[pv] B(pu,pv) / NP
// (CONJ: its conjugate, for the adjoint).
template <class TL, bool CONJ>
struct PropOp {
  const float2* h;
  const int* fsq;
  int blT;
  __device__ void operator()(int pu, int pv, float2& v) const {
    // fsq of the row slot from its index (no table read); the column
    // factor h[pv] / NP is common to a column task's slots
    const int fu = TL::freq(TL::nat(pu));
    const bool keep = blT < 0 || fu * fu + fsq[pv] <= blT;
    const float2 hh = cmul(h[pu], cscale(h[pv], 1.0f / (float)TL::NP));
    const float2 w = CONJ ? cmulc(v, hh) : cmul(v, hh);
    v = keep ? w : make_float2(0.f, 0.f);
  }
};

// One full forward pass of item (j, k) from the shifted probe to the far
// field.  WAVES: the entry wave psi_s of every slice is written to `waves`
// (natural order, NP per slice, format Var<V>::prec); ePIE variants also
// record max |psi_s|^2 per slice in D.wmax.  On return the column layout
// holds F(phi_{S-1}) after its column s1 stage: the caller applies the last
// column s2 (far field) with its own pointwise op.
template <class TL, int V, bool WAVES>
__device__ void forward_chain(const Smem<TL>& sm, int rank, const ProblemDesc& D, const ItemGeo& g,
                              char* waves) {
  constexpr int N = TL::N;
  constexpr int PREC = Var<V>::prec;
  constexpr bool WMAX = Var<V>::epie;
  const float inv = 1.0f / (float)TL::NP;
  const float2* Ph = D.Phat + (size_t)g.k * TL::NP;
  const float2* rY = sm.rampY;
  const float2* rX = sm.rampX;
  // psi_0 = F^-1[ramp . F P_k]: column s2' straight from the stored spectrum
  TL::template col_contig<false, false, true>(
      sm.wave, sm.twC, rank,
      [&](int pu, int pv) { return cscale(cmul(cmul(__ldg(Ph + pu * N + pv), rY[pu]), rX[pv]), inv); },
      NoOp{});
  __syncthreads();
  TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
#pragma unroll 1
  for (int s = 0; s < D.S; ++s) {
    if (s + 1 < D.S) load_chirp<TL>(sm.chirp + (s & 1) * N, D.Hc + (size_t)s * N);
    const float2* Os = D.O + (size_t)s * D.H * D.W + (size_t)g.ny * D.W + g.nx;
    char* wv = WAVES ? waves + (size_t)s * TL::NP * Var<V>::wave_bytes : nullptr;
    const int W = D.W;
    // row s1' (finishing psi_s) -> store psi_s -> transmit -> row s1
    float lm = 0.f;
    float* ils = Var<V>::lsq_dir ? D.lsq_il + (size_t)s * D.H * D.W + (size_t)g.ny * D.W + g.nx : nullptr;
    TL::template row_strided<true, true>(sm.wave, sm.twS, rank, NoLoad{}, PreO{Os, W},
                                         [&](int r, int c, float2& v, const float2& o) {
                                           if constexpr (WAVES) wave_put<PREC>(wv, r * N + c, v);
                                           if constexpr (WMAX) lm = fmaxf(lm, cabs2(v));
                                           if constexpr (Var<V>::lsq_dir) red_add1(ils + (size_t)r * W + c, cabs2(v));
                                           v = cmul(v, o);
                                         });
    if constexpr (WMAX) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lm = fmaxf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
      // non-negative floats order like their bit patterns
      if ((threadIdx.x & 31) == 0) atomicMax(D.wmax + ((size_t)g.j * D.K + g.k) * D.S + s, __float_as_uint(lm));
    }
    TL::row_sync();  // the row -> column stage stays within rows until its exchange
    TL::forward_mid(sm.wave, sm.twS, sm.twC, rank);
    if (s + 1 < D.S) {
      TL::template col_contig<true, true, true>(sm.wave, sm.twC, rank, NoLoad{},
                                                PropOp<TL, false>{sm.chirp + (s & 1) * N, sm.fsq, D.blT});
      __syncthreads();
      TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
    }
  }
}

// Backward pass of item (j, k) from g_phi_{S-1} (row layout, pending row
// s1') to the probe spectrum gradient.  psi_s are read from `waves`
// (format Var<V>::prec).  ePIE variants scale the object term by
// 1 / max|psi_s|^2 and the incident-wave term by 1 / max|O_s|^2 (§3.3.1).
template <class TL, int V>
__device__ void adjoint_chain(const Smem<TL>& sm, int rank, const ProblemDesc& D, const ItemGeo& g,
                              const char* waves) {
  constexpr int N = TL::N;
#pragma unroll 1
  for (int s = D.S - 1; s >= 0; --s) {
    if (s > 0) load_chirp<TL>(sm.chirp + (s & 1) * N, D.Hc + (size_t)(s - 1) * N);
    const size_t ooff = (size_t)s * D.H * D.W + (size_t)g.ny * D.W + g.nx;
    const float2* Os = D.O + ooff;
    float2* gOs = D.gO + ooff;
    const char* wv = waves + (size_t)s * TL::NP * Var<V>::wave_bytes;
    const int W = D.W;
    // row s1' (finishing g_phi_s) -> object gradient, g_psi_s = conj(O) g_phi -> row s1
    if constexpr (Var<V>::lsq_step) {
      // LSQML step sizes: with chi_s = g_phi_s (the exit-plane update) and
      // q = dO_s psi_s, sum Re(chi conj q) and |q|^2 over the window; at the
      // entry slice also with q = O_0 S_j dP_k (the shifted probe direction,
      // kept after this mode's entry waves)
      const float2* dOs = D.lsq_dO + ooff;
      const float2* sdp = reinterpret_cast<const float2*>(waves + (size_t)D.S * TL::NP * Var<V>::wave_bytes);
      float num = 0.f, den = 0.f, nump = 0.f, denp = 0.f;
      TL::template row_strided<true, true>(sm.wave, sm.twS, rank, NoLoad{}, PrePsiO<0>{wv, N, Os, W},
                                           [&](int r, int c, float2& v, const PsiO& p) {
                                             const float2 q = cmul(__ldg(dOs + (size_t)r * W + c), p.psi);
                                             num = fmaf(v.x, q.x, fmaf(v.y, q.y, num));
                                             den += cabs2(q);
                                             if (s == 0) {
                                               const float2 qp = cmul(p.o, sdp[r * N + c]);
                                               nump = fmaf(v.x, qp.x, fmaf(v.y, qp.y, nump));
                                               denp += cabs2(qp);
                                             }
                                             v = cconjmul(p.o, v);
                                           });
      const double sn = warp_sum((double)num), sd = warp_sum((double)den);
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(D.lsq_num + (size_t)g.j * D.S + s, sn);
        atomicAdd(D.lsq_den + (size_t)g.j * D.S + s, sd);
      }
      if (s == 0) {
        const double pn = warp_sum((double)nump), pd = warp_sum((double)denp);
        if ((threadIdx.x & 31) == 0) {
          atomicAdd(D.lsq_numP + g.j, pn);
          atomicAdd(D.lsq_denP + g.j, pd);
        }
        break;  // nothing further of the chain is needed
      }
    } else if constexpr (Var<V>::epie) {
      const float inv_o = 1.0f / fmaxf(__uint_as_float(__ldg(D.omax + s)), FLT_MIN);
      const float inv_p =
          1.0f / fmaxf(__uint_as_float(__ldcg(D.wmax + ((size_t)g.j * D.K + g.k) * D.S + s)), FLT_MIN);
      TL::template row_strided<true, true>(sm.wave, sm.twS, rank, NoLoad{}, PrePsiO<Var<V>::prec>{wv, N, Os, W},
                                           [&](int r, int c, float2& v, const PsiO& p) {
                                             red_add(gOs + (size_t)r * W + c, cscale(cconjmul(p.psi, v), inv_p));
                                             v = cscale(cconjmul(p.o, v), inv_o);
                                           });
    } else if constexpr (Var<V>::det) {
      // this position's patch gradient, summed over the modes in mode order
      // (every element is owned by one thread in every mode: program order)
      float2* pg = D.det_gO + ((size_t)g.j * D.S + s) * TL::NP;
      const bool first = g.k == 0;
      TL::template row_strided<true, true>(sm.wave, sm.twS, rank, NoLoad{}, PrePsiO<0>{wv, N, Os, W},
                                           [&](int r, int c, float2& v, const PsiO& p) {
                                             const float2 t = cconjmul(p.psi, v);
                                             float2* q = pg + r * N + c;
                                             *q = first ? t : cadd(*q, t);
                                             v = cconjmul(p.o, v);
                                           });
    } else {
      TL::template row_strided<true, true>(sm.wave, sm.twS, rank, NoLoad{}, PrePsiO<Var<V>::prec>{wv, N, Os, W},
                                           [&](int r, int c, float2& v, const PsiO& p) {
                                             red_add(gOs + (size_t)r * W + c, cconjmul(p.psi, v));
                                             v = cconjmul(p.o, v);
                                           });
    }
    TL::row_sync();  // the row -> column stage stays within rows until its exchange
    TL::forward_mid(sm.wave, sm.twS, sm.twC, rank);
    if (s > 0) {
      TL::template col_contig<true, true, true>(sm.wave, sm.twC, rank, NoLoad{},
                                                PropOp<TL, true>{sm.chirp + (s & 1) * N, sm.fsq, D.blT});
      __syncthreads();
      TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
    } else {
      // F g_psi_0 -> conj(ramp) -> accumulate the probe spectrum gradient.
      // Position gradient (through the ramp only; the patch origin is
      // piecewise constant): dL/d(delta_y) = 2 pi / (N NP) sum f_u Im(w),
      // w = conj(F g_psi_0) ramp F P, likewise for x with f_v.
      float2* gP = D.gPhat + (size_t)g.k * TL::NP;
      float2* gPj = Var<V>::det ? D.det_gP + ((size_t)g.j * D.K + g.k) * TL::NP : nullptr;
      const float2* Ph = D.Phat + (size_t)g.k * TL::NP;
      const float2* rY = sm.rampY;
      const float2* rX = sm.rampX;
      const bool want_pos = D.gpos != nullptr;
      float sy = 0.f, sx = 0.f;
      TL::template col_contig<true, true, false>(sm.wave, sm.twC, rank, NoLoad{}, [&](int pu, int pv, float2& v) {
        const float2 ramp = cmul(rY[pu], rX[pv]);
        if constexpr (Var<V>::det) gPj[pu * N + pv] = cmulc(v, ramp);
        else red_add(gP + pu * N + pv, cmulc(v, ramp));
        if (want_pos) {
          const float w = cconjmul(v, cmul(ramp, __ldg(Ph + pu * N + pv))).y;
          sy = fmaf((float)TL::freq(TL::nat(pu)), w, sy);
          sx = fmaf((float)TL::freq(TL::nat(pv)), w, sx);
        }
      });
      if (want_pos) {
        double dy = sy, dx = sx;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dy += __shfl_xor_sync(0xffffffffu, dy, o);
          dx += __shfl_xor_sync(0xffffffffu, dx, o);
        }
        if ((threadIdx.x & 31) == 0) {
          const double sc = 2.0 * 3.14159265358979323846 / ((double)N * (double)TL::NP);
          atomicAdd(D.gpos + 2 * (size_t)g.j, sc * dy);
          atomicAdd(D.gpos + 2 * (size_t)g.j + 1, sc * dx);
        }
      }
    }
  }
}

template <class TL>
__device__ __forceinline__ int cluster_id() { return blockIdx.x / TL::G; }
template <class TL>
__device__ __forceinline__ int n_clusters() { return gridDim.x / TL::G; }
template <class TL>
__device__ __forceinline__ int my_rank() {
  if constexpr (TL::G > 1) return (int)cluster_rank(); else return 0;
}

// ---------------------------------------------------------------------------
// Forward: far field A = F(phi_{S-1}) (unnormalised, spectral slot order) of
// every item; optionally every entry wave psi_s (STORE).
template <class TL, bool STORE, int V>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_forward(const __grid_constant__ LaunchArgs L) {
  extern __shared__ float4 smem_raw[];
  Smem<TL> sm(smem_raw);
  const int rank = my_rank<TL>();
  TL::init_tables(sm.twS, sm.twC, sm.fsq);
  constexpr int N = TL::N;
#pragma unroll 1
  for (int it = cluster_id<TL>(); it < L.total; it += n_clusters<TL>()) {
    const int item = L.order ? __ldg(L.order + it / L.d[0].K) * L.d[0].K + it % L.d[0].K : it;
    // the partner CTAs must be done with the previous item before remote
    // writes of this one can land in their exchange buffers
    TL::sync_cluster();
    const ProblemDesc& D = find_desc(L, item);
    const ItemGeo g = item_geo<TL>(D, item);
    if (!g.ok) {
      if (threadIdx.x == 0 && rank == 0) atomicOr(L.status, PTYCHO_STATUS_OUT_OF_BOUNDS);
      continue;
    }
    __syncthreads();
    make_ramps<TL>(sm.rampY, sm.rampX, g.dy, g.dx);
    __syncthreads();
    char* waves = STORE ? D.waves + ((size_t)g.j * D.K + g.k) * D.S * TL::NP * Var<V>::wave_bytes : nullptr;
    forward_chain<TL, V, STORE>(sm, rank, D, g, waves);
    float2* Aout = D.A + ((size_t)g.j * D.K + g.k) * TL::NP;
    TL::template col_contig<true, true, false>(sm.wave, sm.twC, rank, NoLoad{},
                                               [&](int pu, int pv, float2& v) { Aout[pu * N + pv] = v; });
  }
  // no CTA leaves while its partner may still be sending to it
  TL::sync_cluster();
}

// Adjoint.  STORE: psi_s come from the forward's store; the seed is
// w . A from global memory.  Otherwise the forward is recomputed here with
// psi_s written to this cluster's slot, and the far field is turned into
// the seed without leaving shared memory.
template <class TL, bool STORE, int V>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_adjoint(const __grid_constant__ LaunchArgs L) {
  extern __shared__ float4 smem_raw[];
  Smem<TL> sm(smem_raw);
  const int rank = my_rank<TL>();
  TL::init_tables(sm.twS, sm.twC, sm.fsq);
  constexpr int N = TL::N;
#pragma unroll 1
  for (int it = cluster_id<TL>(); it < L.total; it += n_clusters<TL>()) {
    const int item = L.order ? __ldg(L.order + it / L.d[0].K) * L.d[0].K + it % L.d[0].K : it;
    // the partner CTAs must be done with the previous item before remote
    // writes of this one can land in their exchange buffers
    TL::sync_cluster();
    const ProblemDesc& D = find_desc(L, item);
    const ItemGeo g = item_geo<TL>(D, item);
    if (!g.ok) {
      if (threadIdx.x == 0 && rank == 0) atomicOr(L.status, PTYCHO_STATUS_OUT_OF_BOUNDS);
      continue;
    }
    __syncthreads();
    make_ramps<TL>(sm.rampY, sm.rampX, g.dy, g.dx);
    __syncthreads();
    const float* wj = D.w + (size_t)g.j * TL::NP;
    const char* waves;
    if constexpr (STORE) {
      waves = D.waves + ((size_t)g.j * D.K + g.k) * D.S * TL::NP * Var<V>::wave_bytes;
      const float2* Aj = D.A + ((size_t)g.j * D.K + g.k) * TL::NP;
      TL::template col_contig<false, false, true>(
          sm.wave, sm.twC, rank, [&](int pu, int pv) { return cscale(Aj[pu * N + pv], wj[pu * N + pv]); },
          NoOp{});
      __syncthreads();
    } else {
      char* slot = L.slots + (size_t)cluster_id<TL>() * L.slot_stride;
      waves = slot;
      forward_chain<TL, V, true>(sm, rank, D, g, slot);
      TL::template col_contig<true, true, true>(sm.wave, sm.twC, rank, NoLoad{},
                                                [&](int pu, int pv, float2& v) { v = cscale(v, wj[pu * N + pv]); });
      __syncthreads();
    }
    TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
    adjoint_chain<TL, V>(sm, rank, D, g, waves);
  }
  // no CTA leaves while its partner may still be sending to it
  TL::sync_cluster();
}

// Work queue of the position-major launch (PosArgs::queue): rank 0's thread
// 0 claims the next entry of the processing order for its cluster and stores
// it in the claim word of every CTA of the cluster (visible to all of them
// after the next cluster barrier).
template <class TL>
__device__ __forceinline__ void claim_next(int* claim, unsigned* queue, int rank) {
  if (rank == 0 && threadIdx.x == 0) {
    const int v = (int)atomicAdd(queue, 1u);
    if constexpr (TL::G > 1) {
      const uint32_t a = smem_u32(claim);
#pragma unroll
      for (int r = 0; r < TL::G; ++r) st_cluster_s32(cluster_map(a, (uint32_t)r), v);
    } else {
      *claim = v;
    }
  }
}

// One scan position of the position-major kernel: entry `it` of the
// launch's processing order, run by the cluster that holds slot, Ab and Ib
// (see k_adjoint_pos).
template <class TL, int V>
__device__ __forceinline__ void adjoint_position(Smem<TL>& sm, const LaunchArgs& L, const PosArgs& F, int rank,
                                                 int it, char* slot, float2* Ab, float* Ib) {
  constexpr int N = TL::N;
  constexpr float inv = 1.0f / (float)TL::NP;
  const int jg = F.order ? __ldg(F.order + it) : it;
  // position j of problem D (item0: its first position in the launch)
  const ProblemDesc& D = find_desc(L, jg);
  const int j = jg - D.item0;
  const int K = D.K;
  // one mode's entry waves (and, in the LSQML step pass, its shifted probe direction)
  const size_t wstride = (size_t)(D.S + Var<V>::extra_waves) * TL::NP * Var<V>::wave_bytes;
  ItemGeo g = item_geo<TL>(D, D.item0 + j * K);
  if (!g.ok) {  // every mode of this position skips it
    if (threadIdx.x == 0 && rank == 0) atomicOr(L.status, PTYCHO_STATUS_OUT_OF_BOUNDS);
    // every CTA has read the claim word before the next claim is stored
    TL::sync_cluster();
    return;
  }
  make_ramps<TL>(sm.rampY, sm.rampX, g.dy, g.dx);
  __syncthreads();
  const float* E = D.Iexp + (size_t)g.jj * TL::NP;
  float lsum = 0.f;
#pragma unroll 1
  for (int k = 0; k < K; ++k) {
    if (k) TL::sync_cluster();
    g.k = k;
    if constexpr (Var<V>::lsq_step) {
      // S_j dP_k = F^-1[ramp . F dP_k], natural order, after the mode's entry waves
      float2* out = reinterpret_cast<float2*>(slot + k * wstride + (size_t)D.S * TL::NP * Var<V>::wave_bytes);
      const float2* dPh = D.lsq_dPhat + (size_t)k * TL::NP;
      const float2* rY = sm.rampY;
      const float2* rX = sm.rampX;
      TL::template col_contig<false, false, true>(
          sm.wave, sm.twC, rank,
          [&](int pu, int pv) { return cscale(cmul(cmul(__ldg(dPh + pu * N + pv), rY[pu]), rX[pv]), inv); },
          NoOp{});
      __syncthreads();
      TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
      TL::template row_strided<true, false>(sm.wave, sm.twS, rank, NoLoad{}, NoPre{},
                                            [&](int r, int c, float2& v, const NoPre::type&) { out[r * N + c] = v; });
      TL::sync_cluster();
    }
    forward_chain<TL, V, true>(sm, rank, D, g, slot + k * wstride);
    float2* Ak = Ab + (size_t)k * TL::NP;
    const bool first = k == 0, last = k + 1 == K;
    TL::template col_contig<true, true, false>(sm.wave, sm.twC, rank, NoLoad{}, [&](int pu, int pv, float2& v) {
      const int p = pu * N + pv;
      Ak[p] = v;
      float I = cabs2(v) * inv;
      if (!first) I += Ib[p];
      if (!last) {
        Ib[p] = I;
      } else {
        float l, dl;
        noise_model(D.model, D.eps, D.c, I, __ldg(E + TL::nat(pu) * N + TL::nat(pv)), l, dl);
        lsum += l;
        Ib[p] = 2.0f * dl * inv;
      }
    });
  }
  {
    double sd = lsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(D.lpart + j, sd);
  }
#pragma unroll 1
  for (int k = 0; k < K; ++k) {
    TL::sync_cluster();
    g.k = k;
    const float2* Ak = Ab + (size_t)k * TL::NP;
    TL::template col_contig<false, false, true>(
        sm.wave, sm.twC, rank,
        [&](int pu, int pv) {
          const int p = pu * N + pv;
          return cscale(Ak[p], Ib[p]);
        },
        NoOp{});
    __syncthreads();
    TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
    adjoint_chain<TL, V>(sm, rank, D, g, slot + k * wstride);
  }
  if constexpr (Var<V>::lsq_step) {
    // every mode has added its sums: step-weighted illumination
    // alpha_{s,j} sum_k |psi_{s,k}|^2 over this CTA's rows of the window
    TL::sync_cluster();
    const int W = D.W;
#pragma unroll 1
    for (int s = 0; s < D.S; ++s) {
      const double num = __ldcg(D.lsq_num + (size_t)j * D.S + s), den = __ldcg(D.lsq_den + (size_t)j * D.S + s);
      const float a = den + (double)F.gamma > 0.0 ? (float)(num / (den + (double)F.gamma)) : 0.f;
      float* aws = D.lsq_aw + (size_t)s * D.H * D.W + (size_t)g.ny * D.W + g.nx;
      for (int e = threadIdx.x; e < TL::ROWS * N; e += TL::T) {
        const int r = rank * TL::ROWS + e / N, c = e % N;
        float w = 0.f;
        for (int k = 0; k < K; ++k)
          w += cabs2(__ldcg(reinterpret_cast<const float2*>(slot + k * wstride + (size_t)s * TL::NP * 8) + r * N + c));
        red_add1(aws + (size_t)r * W + c, a * w);
      }
    }
  }
}

// Loss + adjoint with the entry waves recomputed, one cluster per scan
// position (position-major, one launch per step, no waits between
// clusters; the positions of several problems of one window size may share
// a launch).  For position j the cluster runs the forward pass of every
// mode k (entry waves to part k of its slot, far field A_k to its scratch,
// the intensity summed over modes in its scratch), applies the noise model
// to the mode sum (loss into lpart[j], seed weight 2 l'(I) / NP in place of
// I), then runs the backward pass of every mode from the seed w A_k.  Every
// pixel of the scratch is written and read back by the same thread (the
// column stage's task mapping), so the scratch needs no synchronisation
// beyond program order.
//
// Assignment of positions to clusters.  Without QUEUE (launches of one
// problem, whose positions all cost the same) cluster c takes entries c,
// c + clusters, ... of the processing order.  With QUEUE (launches that mix
// problems: positions cost S slices times K modes of their own problem)
// cluster c takes entry c first and then claims the next entry from the
// launch's work queue whenever it finishes a position, so that clusters
// finishing early take more.  Claims are made at the end of a position
// rather than ahead of it: an early claim would take work from clusters
// that have not started yet.  (The queue's loop state costs the kernel 9
// registers, and launches of one problem 1.2 % of their time, so they keep
// the static assignment.)
template <class TL, int V, bool QUEUE>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_adjoint_pos(const __grid_constant__ LaunchArgs L,
                                                                 const __grid_constant__ PosArgs F) {
  extern __shared__ float4 smem_raw[];
  Smem<TL> sm(smem_raw);
  const int rank = my_rank<TL>();
  TL::init_tables(sm.twS, sm.twC, sm.fsq);
  const int cid = cluster_id<TL>();
  char* slot = L.slots + (size_t)cid * L.slot_stride;
  float2* Ab = F.Abuf + (size_t)cid * F.astride;
  float* Ib = F.Ibuf + (size_t)cid * TL::NP;
  pdl_wait();
  if constexpr (!QUEUE) {
#pragma unroll 1
    for (int it = cid; it < L.total; it += n_clusters<TL>()) {
      // the partner CTAs are done with the previous position
      TL::sync_cluster();
      adjoint_position<TL, V>(sm, L, F, rank, it, slot, Ab, Ib);
    }
    pdl_trigger();
    // no CTA leaves while its partner may still be sending to it
    TL::sync_cluster();
  } else {
    // claim word: written at the end of a position, read after the next
    // cluster barrier, written again only after at least one more (every
    // position's work holds one: the backward pass of each mode starts with
    // it, and a skipped position takes one)
    __shared__ int claim;
    const bool queued = L.total > n_clusters<TL>();
    int it = cid;  // entry of the processing order; < 0: read the claim
#pragma unroll 1
    for (;;) {
      // also: the partner CTAs are done with the previous position
      TL::sync_cluster();
      if (it < 0) it = n_clusters<TL>() + claim;
      if (it >= L.total) break;
      adjoint_position<TL, V>(sm, L, F, rank, it, slot, Ab, Ib);
      // claim the next entry (or leave when every position has its cluster)
      if (queued) {
        claim_next<TL>(&claim, F.queue, rank);
        it = -1;
      } else {
        it = L.total;
      }
    }
    pdl_trigger();
    // no CTA leaves while its partner may still be sending to it
    TL::sync_cluster();
    // every cluster made its last claim before counting itself out, so the
    // last one out can reset the queue for the next launch
    if (queued && rank == 0 && threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(F.queue + 1, 1u) == (unsigned)n_clusters<TL>() - 1u) {
        atomicExch(F.queue, 0u);
        atomicExch(F.queue + 1, 0u);
      }
    }
  }
}

// Probe spectra P^_k = F P_k in spectral slot order (one item per mode).
template <class TL>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_probe_spectrum(const float2* __restrict__ P, float2* __restrict__ Phat, int K) {
  extern __shared__ float4 smem_raw[];
  Smem<TL> sm(smem_raw);
  const int rank = my_rank<TL>();
  TL::init_tables(sm.twS, sm.twC, sm.fsq);
  __syncthreads();
  pdl_wait();
  constexpr int N = TL::N;
#pragma unroll 1
  for (int k = cluster_id<TL>(); k < K; k += n_clusters<TL>()) {
    const float2* Pk = P + (size_t)k * TL::NP;
    float2* out = Phat + (size_t)k * TL::NP;
    TL::sync_cluster();
    TL::template row_strided<false, true>(sm.wave, sm.twS, rank,
                                          [&](int r, int c) { return Pk[r * N + c]; }, NoPre{}, NoOp4{});
    __syncthreads();
    TL::forward_mid(sm.wave, sm.twS, sm.twC, rank);
    TL::template col_contig<true, true, false>(sm.wave, sm.twC, rank, NoLoad{},
                                               [&](int pu, int pv, float2& v) { out[pu * N + pv] = v; });
  }
  pdl_trigger();
  // no CTA leaves while its partner may still be sending to it
  TL::sync_cluster();
}

// Probe gradient g_P_k = F^-1 g_P^_k (natural order); ACC adds to gP.
template <class TL>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_probe_grad(const float2* __restrict__ gPhat, float2* __restrict__ gP, int K, int acc) {
  extern __shared__ float4 smem_raw[];
  Smem<TL> sm(smem_raw);
  const int rank = my_rank<TL>();
  TL::init_tables(sm.twS, sm.twC, sm.fsq);
  __syncthreads();
  pdl_wait();
  constexpr int N = TL::N;
  const float inv = 1.0f / (float)TL::NP;
#pragma unroll 1
  for (int k = cluster_id<TL>(); k < K; k += n_clusters<TL>()) {
    const float2* src = gPhat + (size_t)k * TL::NP;
    float2* out = gP + (size_t)k * TL::NP;
    TL::sync_cluster();
    TL::template col_contig<false, false, true>(sm.wave, sm.twC, rank,
                                                [&](int pu, int pv) { return src[pu * N + pv]; }, NoOp{});
    __syncthreads();
    TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
    TL::template row_strided<true, false>(sm.wave, sm.twS, rank, NoLoad{}, NoPre{},
                                          [&](int r, int c, float2& v, const NoPre::type&) {
                                            const float2 x = cscale(v, inv);
                                            out[r * N + c] = acc ? cadd(out[r * N + c], x) : x;
                                          });
  }
  // no CTA leaves while its partner may still be sending to it
  TL::sync_cluster();
}

// Fused end of a gradient step (TailArgs), single-CTA tiles only.  Blocks
// [0, K): the probe gradient of mode k through the tile (inverse FFT of
// g_P^_k / NP), then Adam on P_k straight from the real-space stage; blocks
// [K, gridDim.x): Adam on the object, grid-stride.  Every block writes the
// FP64 |g|^2 of the elements it read to normp[block]; the last block to
// finish sums the loss partials and the norm partials in a fixed order
// (deterministic for a fixed grid).  Same arithmetic as k_probe_grad,
// k_adam and k_finalize.
constexpr int kTailBatch = 8;
template <class TL>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_step_tail(const __grid_constant__ TailArgs A) {
  static_assert(TL::G == 1, "single-CTA tiles");
  extern __shared__ float4 smem_raw[];
  __shared__ double sh[32];
  __shared__ unsigned ticket;
  constexpr int N = TL::N;
  double acc = 0.0;
  if ((int)blockIdx.x < A.K) {
    Smem<TL> sm(smem_raw);
    TL::init_tables(sm.twS, sm.twC, sm.fsq);
    __syncthreads();
    pdl_wait();
    const float bc1 = A.bcd ? A.bcd[0] : A.bc1;  // written by an earlier kernel: after the wait
    const float bc2 = A.bcd ? A.bcd[1] : A.bc2;
    const int k = blockIdx.x;
    float2* src = A.gPhat + (size_t)k * TL::NP;
    TL::template col_contig<false, false, true>(sm.wave, sm.twC, 0, [&](int pu, int pv) { return src[pu * N + pv]; },
                                                NoOp{});
    __syncthreads();
    // g_P^_k is in shared memory now: clear it for the next step's accumulation
    for (int e = threadIdx.x; e < TL::NP; e += TL::T) src[e] = make_float2(0.f, 0.f);
    TL::inverse_tail(sm.wave, sm.twS, sm.twC, 0);
    // last inverse stage in place (each task writes back the natural-order
    // samples of the slots it read), then the Adam update over the mode in
    // natural order with every thread, so that its global accesses coalesce
    TL::template row_strided<true, false>(sm.wave, sm.twS, 0, NoLoad{}, NoPre{},
                                          [&](int r, int c, float2& v, const NoPre::type&) {
                                            sm.wave[TL::rslot(0, c / TL::ROWS, r, c % TL::ROWS)] = v;
                                          });
    __syncthreads();
    const float inv = 1.0f / (float)TL::NP;
    float2* Pk = A.P + (size_t)k * TL::NP;
    float2* mk = A.mP + (size_t)k * TL::NP;
    float* vk = A.vP + (size_t)k * TL::NP;
    // kTailBatch elements per thread in flight: all loads of a batch are
    // issued before its stores
    for (int e0 = threadIdx.x; e0 < TL::NP; e0 += kTailBatch * TL::T) {
      float2 g[kTailBatch], z[kTailBatch], m[kTailBatch];
      float v[kTailBatch];
#pragma unroll
      for (int u = 0; u < kTailBatch; ++u) {
        const int e = e0 + u * TL::T;
        if (e < TL::NP) {
          const int r = e / N, c = e % N;
          g[u] = cscale(sm.wave[TL::rslot(0, c / TL::ROWS, r, c % TL::ROWS)], inv);
          if (A.update_probe) {
            z[u] = Pk[e];
            m[u] = mk[e];
            v[u] = vk[e];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kTailBatch; ++u) {
        const int e = e0 + u * TL::T;
        if (e < TL::NP) {
          acc += (double)g[u].x * g[u].x + (double)g[u].y * g[u].y;
          if (A.update_probe) {
            adam_math(z[u], m[u], v[u], g[u], A.lrP, A.b1, A.b2, A.eps, bc1, bc2);
            Pk[e] = z[u];
            mk[e] = m[u];
            vk[e] = v[u];
          }
        }
      }
    }
  } else {
    pdl_wait();
    const float bc1 = A.bcd ? A.bcd[0] : A.bc1;
    const float bc2 = A.bcd ? A.bcd[1] : A.bc2;
    const long long stride = (long long)(gridDim.x - A.K) * TL::T;
    for (long long e0 = (long long)(blockIdx.x - A.K) * TL::T + threadIdx.x; e0 < A.nO; e0 += kTailBatch * stride) {
      float2 g[kTailBatch], z[kTailBatch], m[kTailBatch];
      float v[kTailBatch];
#pragma unroll
      for (int u = 0; u < kTailBatch; ++u) {
        const long long e = e0 + u * stride;
        if (e < A.nO) {
          g[u] = A.gO[e];
          z[u] = A.O[e];
          m[u] = A.mO[e];
          v[u] = A.vO[e];
        }
      }
#pragma unroll
      for (int u = 0; u < kTailBatch; ++u) {
        const long long e = e0 + u * stride;
        if (e < A.nO) {
          acc += (double)g[u].x * g[u].x + (double)g[u].y * g[u].y;
          adam_math(z[u], m[u], v[u], g[u], A.lrO, A.b1, A.b2, A.eps, bc1, bc2);
          A.gO[e] = make_float2(0.f, 0.f);
          A.O[e] = z[u];
          A.mO[e] = m[u];
          A.vO[e] = v[u];
        }
      }
    }
  }
  pdl_trigger();
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) A.normp[blockIdx.x] = t;
  // last block done: the final sums, in a fixed order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(A.counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < A.nl; i += TL::T) a += __ldcg(A.lossp + i);
  for (int i = threadIdx.x; i < (int)gridDim.x; i += TL::T) b += __ldcg(A.normp + i);
  const double ta = block_sum(a, sh);
  const double tb = block_sum(b, sh);
  for (int i = threadIdx.x; i < A.nz; i += TL::T) A.lossp[i] = 0.0;
  if (threadIdx.x == 0) {
    A.stats[0] = ta;
    A.stats[1] = sqrt(tb);
    *A.counter = 0u;
  }
}

// Self-test of the exchange's bounded wait (tests): every CTA of one cluster
// waits for a block that nothing sends, with a short poll limit, so each
// wait gives up and flags the time-out; the CTAs then leave together.
template <class TL>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_exchange_timeout_probe() {
  extern __shared__ float4 smem_raw[];
  Smem<TL> sm(smem_raw);
  TL::init_tables(sm.twS, sm.twC, sm.fsq);
  TL::sync_cluster();
  if constexpr (TL::XB) TL::exchange_wait(sm.wave, 0, 1u << 12);
  TL::sync_cluster();
}

// Stand-alone 2-D DFT of natural-order arrays through the tile (tests).
// dir < 0: unnormalised forward; dir > 0: unnormalised inverse.
template <class TL>
__global__ void __launch_bounds__(TL::T, TL::MINB) k_fft_debug(const float2* __restrict__ in, float2* __restrict__ out, int count, int dir) {
  extern __shared__ float4 smem_raw[];
  Smem<TL> sm(smem_raw);
  const int rank = my_rank<TL>();
  TL::init_tables(sm.twS, sm.twC, sm.fsq);
  __syncthreads();
  constexpr int N = TL::N;
#pragma unroll 1
  for (int b = cluster_id<TL>(); b < count; b += n_clusters<TL>()) {
    const float2* x = in + (size_t)b * TL::NP;
    float2* y = out + (size_t)b * TL::NP;
    TL::sync_cluster();
    if (dir < 0) {
      TL::template row_strided<false, true>(sm.wave, sm.twS, rank, [&](int r, int c) { return x[r * N + c]; },
                                            NoPre{}, NoOp4{});
      __syncthreads();
      TL::forward_mid(sm.wave, sm.twS, sm.twC, rank);
      TL::template col_contig<true, true, false>(sm.wave, sm.twC, rank, NoLoad{}, [&](int pu, int pv, float2& v) {
        y[TL::nat(pu) * N + TL::nat(pv)] = v;
      });
    } else {
      TL::template col_contig<false, false, true>(
          sm.wave, sm.twC, rank, [&](int pu, int pv) { return x[TL::nat(pu) * N + TL::nat(pv)]; }, NoOp{});
      __syncthreads();
      TL::inverse_tail(sm.wave, sm.twS, sm.twC, rank);
      TL::template row_strided<true, false>(sm.wave, sm.twS, rank, NoLoad{}, NoPre{},
                                            [&](int r, int c, float2& v, const NoPre::type&) { y[r * N + c] = v; });
    }
  }
  // no CTA leaves while its partner may still be sending to it
  TL::sync_cluster();
}

}  // namespace ptycho
