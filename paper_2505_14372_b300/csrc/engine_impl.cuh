// Launchers of one tile shape; included once per window size.
#pragma once
#include <algorithm>
#include <type_traits>

#include "elementwise.cuh"
#include "engine.h"
#include "kernels.cuh"

namespace ptycho {

// ALLV: instantiate every Variant (otherwise FP32 gradient kernels only).
template <class TL, bool ALLV = true>
struct Engine {
  // calls f(std::integral_constant<int, V>) for the runtime variant; the
  // LSQML passes exist only for the position-major kernel (MAXV)
  template <int MAXV = kVarEpie, class F>
  static cudaError_t with_variant(int variant, const F& f) {
    if constexpr (ALLV) {
      switch (variant) {
        case kVarF32: return f(std::integral_constant<int, kVarF32>{});
        case kVarF16: return f(std::integral_constant<int, kVarF16>{});
        case kVarBF16: return f(std::integral_constant<int, kVarBF16>{});
        case kVarEpie: return f(std::integral_constant<int, kVarEpie>{});
        case kVarLsqDir:
          if constexpr (MAXV >= kVarLsqDir) return f(std::integral_constant<int, kVarLsqDir>{});
          else return cudaErrorNotSupported;
        case kVarLsqStep:
          if constexpr (MAXV >= kVarLsqStep) return f(std::integral_constant<int, kVarLsqStep>{});
          else return cudaErrorNotSupported;
        case kVarDet:
          if constexpr (MAXV >= kVarDet) return f(std::integral_constant<int, kVarDet>{});
          else return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
      }
    } else {
      if (variant != kVarF32) return cudaErrorNotSupported;
      return f(std::integral_constant<int, kVarF32>{});
    }
  }

  // PDL: launch with programmatic stream serialization (the kernel waits
  // with griddepcontrol.wait before reading what earlier kernels wrote)
  template <class K>
  static cudaError_t launch_ex(K kernel, int clusters, bool pdl, cudaStream_t s, auto... args) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * TL::G), 1, 1);
    cfg.blockDim = dim3(TL::T, 1, 1);
    cfg.dynamicSmemBytes = TL::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int n = 0;
    if (TL::G > 1) {
      attr[n].id = cudaLaunchAttributeClusterDimension;
      attr[n].val.clusterDim.x = TL::G;
      attr[n].val.clusterDim.y = 1;
      attr[n].val.clusterDim.z = 1;
      ++n;
    }
    if (pdl) {
      attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[n].val.programmaticStreamSerializationAllowed = 1;
      ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    count_launch();
    return cudaLaunchKernelEx(&cfg, kernel, args...);
  }
  template <class K>
  static cudaError_t launch(K kernel, int clusters, cudaStream_t s, auto... args) {
    return launch_ex(kernel, clusters, false, s, args...);
  }

  template <class K>
  static int resident(K kernel) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::SMEM) != cudaSuccess)
      return std::max(1, nsm / TL::G);
    if constexpr (TL::G > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(nsm / TL::G * TL::G), 1, 1);
      cfg.blockDim = dim3(TL::T, 1, 1);
      cfg.dynamicSmemBytes = TL::SMEM;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = TL::G;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return std::max(1, nsm / TL::G);
      }
      return n;
    } else {
      int per = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, TL::T, TL::SMEM) != cudaSuccess || per <= 0) {
        cudaGetLastError();
        return nsm;
      }
      return per * nsm;
    }
  }

  static cudaError_t probe_spectrum(const float2* P, float2* Phat, int K, cudaStream_t s) {
    return launch_ex(k_probe_spectrum<TL>, K, true, s, P, Phat, K);
  }
  static cudaError_t forward(const LaunchArgs& L, int clusters, bool store, int variant, cudaStream_t s) {
    // without stored waves the forward writes the far field only (the
    // recomputing adjoint records what ePIE needs itself)
    if (!store) return launch(k_forward<TL, false, kVarF32>, clusters, s, L);
    return with_variant(variant, [&](auto v) { return launch(k_forward<TL, true, decltype(v)::value>, clusters, s, L); });
  }
  static cudaError_t adjoint(const LaunchArgs& L, int clusters, bool store, int variant, cudaStream_t s) {
    return with_variant(variant, [&](auto v) {
      constexpr int V = decltype(v)::value;
      if (store) return launch(k_adjoint<TL, true, V>, clusters, s, L);
      return launch(k_adjoint<TL, false, V>, clusters, s, L);
    });
  }
  static cudaError_t probe_grad(const float2* gPhat, float2* gP, int K, int acc, cudaStream_t s) {
    return launch_ex(k_probe_grad<TL>, K, true, s, gPhat, gP, K, acc);
  }
  static cudaError_t fft_debug(const float2* in, float2* out, int count, int dir, cudaStream_t s) {
    const int cl = std::min(count, resident(k_fft_debug<TL>));
    return launch(k_fft_debug<TL>, std::max(cl, 1), s, in, out, count, dir);
  }
  static cudaError_t modesum(const float2* A, float* I, int B, int K, cudaStream_t s) {
    const long long n = (long long)B * TL::NP;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
    count_launch();
    k_modesum<TL><<<blocks, 256, 0, s>>>(A, I, B, K);
    return cudaGetLastError();
  }
  static cudaError_t loss(const float2* A, const float* Iexp, const int* idx, int npos, int B, int K, int model,
                          float eps, float c, float* w, double* partials, int nblocks, cudaStream_t s) {
    count_launch();
    k_loss<TL><<<nblocks, kRedThreads, 0, s>>>(A, Iexp, idx, npos, B, K, model, eps, c, w, partials);
    return cudaGetLastError();
  }
  static cudaError_t seed(const float* gI, int B, float* w, cudaStream_t s) {
    const long long n = (long long)B * TL::NP;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
    count_launch();
    k_seed<TL><<<blocks, 256, 0, s>>>(gI, B, w);
    return cudaGetLastError();
  }
  // launches that mix problems (positions of different cost) take their
  // positions from the work queue; they run the FP32 gradient variant
  static cudaError_t adjoint_pos(const LaunchArgs& L, const PosArgs& F, int clusters, int variant, cudaStream_t s) {
    if constexpr (ALLV) {  // the tiles that serve requests
      if (L.nd > 1 && variant == kVarF32) {
        if (!F.queue) return cudaErrorInvalidValue;
        return launch_ex(k_adjoint_pos<TL, kVarF32, true>, clusters, true, s, L, F);
      }
    }
    return with_variant<kVarDet>(variant, [&](auto v) {
      return launch_ex(k_adjoint_pos<TL, decltype(v)::value, false>, clusters, true, s, L, F);
    });
  }
  static int resident_pos(int variant) {
    int n = 0;
    with_variant<kVarDet>(variant, [&](auto v) {
      n = resident(k_adjoint_pos<TL, decltype(v)::value, false>);
      return cudaSuccess;
    });
    return n;
  }
  static int resident_clusters(bool adj, bool store, int variant) {
    int n = 0;
    with_variant(variant, [&](auto v) {
      constexpr int V = decltype(v)::value;
      if (adj) n = store ? resident(k_adjoint<TL, true, V>) : resident(k_adjoint<TL, false, V>);
      else n = store ? resident(k_forward<TL, true, V>) : resident(k_forward<TL, false, kVarF32>);
      return cudaSuccess;
    });
    return n;
  }

  // one cluster of the bounded-wait self-test kernel
  static cudaError_t exchange_probe(cudaStream_t s) { return launch(k_exchange_timeout_probe<TL>, 1, s); }

  static unsigned take_exchange_timeouts() {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_exchange_timeouts, sizeof(v)) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    if (v) {
      const unsigned z = 0;
      if (cudaMemcpyToSymbol(g_exchange_timeouts, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
    }
    return v;
  }

  // checked build: index-check bits of this tile's kernels since the last
  // call (read and cleared); always 0 in the normal build
  static unsigned take_check_bits() {
#if PTYCHO_CHECKED
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_bits, sizeof(v)) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    if (v) {
      const unsigned z = 0;
      if (cudaMemcpyToSymbol(g_check_bits, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
    }
    return v;
#else
    return 0;
#endif
  }

  static cudaError_t step_tail(const TailArgs& A, int blocks, cudaStream_t s) {
    if constexpr (TL::G == 1) return launch_ex(k_step_tail<TL>, blocks, true, s, A);
    else return cudaErrorNotSupported;
  }
  // K mode blocks plus enough object blocks for one element per thread, at
  // most one resident wave of them.  Each mode's probe update (and its
  // inverse FFT) runs in one block, so the fused end pays only for small
  // windows: measured, the 64 x 64 step goes 71.6 -> 60.6 us with it, the
  // 128 x 128 step 413 -> 419 us (512 threads) and 411 -> 431 us (1024), so
  // larger tiles keep the separate launches (0: not used).
  static int tail_blocks(long long nO, int K) {
    if constexpr (TL::G == 1 && TL::NP <= 4096) {
      const long long need = std::max(1LL, (nO + TL::T - 1) / TL::T);
      return K + (int)std::min<long long>(need, std::max(1, resident(k_step_tail<TL>)));
    } else {
      return 0;
    }
  }

  static const EngineOps* ops() {
    static const EngineOps o = {TL::N,         TL::G,      TL::T,       TL::R1,      TL::R2,
                                TL::SMEM,      &probe_spectrum, &forward, &adjoint,  &probe_grad,
                                &fft_debug,    &modesum,   &loss,       &seed,       &resident_clusters,
                                &adjoint_pos,  &resident_pos, &take_exchange_timeouts, &exchange_probe, ALLV,
                                &step_tail,    &tail_blocks, &take_check_bits};
    return &o;
  }
};

}  // namespace ptycho
