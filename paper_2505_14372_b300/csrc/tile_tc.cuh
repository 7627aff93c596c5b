// Tensor-core variant of the FFT tile: the same layouts, stages, fusions
// and cluster exchange (in-place results, the off-diagonal block as one bulk
// copy per switch) as Tile, with every R1- and R2-point DFT evaluated by
// tc_dft8 (8 tasks per warp per call) instead of the register butterflies.
// Exposes the interface the kernels use, so the forward/adjoint kernels are
// instantiated unchanged on it.
#pragma once
#include "tc_dft.cuh"
#include "tile.cuh"

namespace ptycho {

// A-fragment tables, [MODE-1][matrix][lane][reg]; matrix 0: R1 forward,
// 1: R1 inverse, 2: R2 forward, 3: R2 inverse (filled once per device by the
// host).  Defined here: only the tensor-core translation unit includes this.
constexpr int kTcTableWords = 32 * 64;
__device__ uint32_t g_tc_tables[kTcModes][4][kTcTableWords];

template <class Base, int MODE>
struct TileTC : Base {
  using B_ = Base;
  static constexpr int N = Base::N, G = Base::G, R1 = Base::R1, R2 = Base::R2, T = Base::T, MINB = Base::MINB;
  static constexpr int NP = Base::NP, ROWS = Base::ROWS, NB = Base::NB, BLK = Base::BLK, WAVE = Base::WAVE;
  static constexpr int TS = Base::TS, TC = Base::TC;
  static constexpr size_t SMEM = Base::SMEM;
  static constexpr bool XB = Base::XB;
  static constexpr int WARPS = T / 32;
  static_assert(G == 1 || XB, "tensor-core tile: single CTA or double-buffered exchange");
  static_assert(TS % 8 == 0 && TC % 8 == 0 && R1 <= 16 && R2 <= 16, "8-task batches of <= 16-point DFTs");

  using Base::cslot;
  using Base::freq;
  using Base::init_tables;
  using Base::nat;
  using Base::perm;
  using Base::rslot;
  using Base::sync_cluster;

  __device__ static const uint32_t* table(int m) { return g_tc_tables[MODE - 1][m]; }
  // this tile's row stages spread rows over all warps
  __device__ static void row_sync() { __syncthreads(); }
  // fragments of the forward R-point matrix; the inverse direction uses
  // the same registers with the off-diagonal signs flipped (tc_dft8 CONJ)
  template <int R>
  __device__ static void load_mat(TcMat<MODE>& M) {
    M.load(table(R == R1 && R1 != R2 ? 0 : 2));
  }

  // ---- row strided ------------------------------------------------------
  template <bool FROM_SMEM, bool TO_SMEM, class Load, class Pre, class Op>
  __device__ static void row_strided(float2* wave, const float2* twS, int rank, const Load& load, const Pre& pre,
                                     const Op& op) {
    const int warp = threadIdx.x >> 5;
    TcMat<MODE> M;
    load_mat<R1>(M);
    auto sl = [&](int id, int e) {
      const int r = id / R2, col = id % R2 + R2 * e;
      return rslot(rank, col / ROWS, r, col % ROWS);
    };
#pragma unroll 1
    for (int q = warp; q < TS / 8; q += WARPS) {
      const int task0 = 8 * q;
      if constexpr (FROM_SMEM) {
        tc_dft8<MODE, R1, true>(
            M, task0, [&](int id, int e) { return wave[sl(id, e)]; },
            [&](int id, int m, float2 v) {
              if constexpr (TO_SMEM) {
                wave[sl(id, m)] = v;
              } else {
                const int r = id / R2, col = id % R2 + R2 * m;
                const int grow = rank * ROWS + r;
                if (chk(grow >= 0 && grow < N && col < N, kChkWindow)) op(grow, col, v, pre(grow, col));
              }
            });
        if constexpr (TO_SMEM) __syncwarp();
      }
      if constexpr (TO_SMEM) {
        tc_dft8<MODE, R1, false>(
            M, task0,
            [&](int id, int e) {
              const int r = id / R2, col = id % R2 + R2 * e;
              const int grow = rank * ROWS + r;
              float2 v = make_float2(0.f, 0.f);
              if (!chk(grow >= 0 && grow < N && col < N, kChkWindow)) return v;
              if constexpr (FROM_SMEM) v = wave[sl(id, e)];
              else v = load(grow, col);
              op(grow, col, v, pre(grow, col));
              return v;
            },
            [&](int id, int k, float2 v) {
              const int n2 = id % R2;
              wave[sl(id, k)] = k ? cmul(v, twS[k * R2 + n2]) : v;
            });
      }
    }
  }

  // ---- row contiguous ---------------------------------------------------
  template <int DIR>
  __device__ static void row_contig(float2* wave, const float2* twC, int rank) {
    const int warp = threadIdx.x >> 5;
    TcMat<MODE> M;
    load_mat<R2>(M);
    auto sl = [&](int id, int e) {
      const int r = id / R1, k1 = id % R1;
      return rslot(rank, k1 / NB, r, R2 * (k1 % NB) + e);
    };
#pragma unroll 1
    for (int q = warp; q < TC / 8; q += WARPS) {
      tc_dft8<MODE, R2, (DIR > 0)>(
          M, 8 * q, [&](int id, int e) { return wave[sl(id, e)]; },
          [&](int id, int m, float2 v) {
            if constexpr (DIR > 0) {
              if (m) v = cmulc(v, twC[m * R1 + id % R1]);
            }
            wave[sl(id, m)] = v;  // in place; the off-diagonal block is sent whole below
          });
    }
    if constexpr (DIR < 0 && G > 1) {
      send_block(wave, rank, 1, 2, 1);
      Base::exchange_wait(wave, 1);
    } else {
      __syncthreads();
    }
  }
  // the layout switch of the 2-CTA tile: every thread's in-place results
  // visible to the copy engine, then the off-diagonal block (slots of block
  // src) goes to the partner's idle buffer dst as one bulk copy counted on
  // its mbarrier `which`
  __device__ static void send_block(float2* wave, int rank, int src, int dst, int which) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) Base::push(wave, rank, src, dst, which, 0, BLK);
  }

  // ---- column strided ---------------------------------------------------
  template <int DIR>
  __device__ static void col_strided(float2* wave, const float2* twS, int rank) {
    const int warp = threadIdx.x >> 5;
    TcMat<MODE> M;
    load_mat<R1>(M);
    auto sl = [&](int id, int e) {
      const int n2 = id / ROWS, cc = id % ROWS;
      return cslot(rank, e / NB, n2 + R2 * (e % NB), cc);
    };
#pragma unroll 1
    for (int q = warp; q < TS / 8; q += WARPS) {
      tc_dft8<MODE, R1, (DIR > 0)>(
          M, 8 * q, [&](int id, int e) { return wave[sl(id, e)]; },
          [&](int id, int m, float2 v) {
            if constexpr (DIR < 0) {
              wave[sl(id, m)] = m ? cmul(v, twS[m * R2 + id / ROWS]) : v;
            } else {
              wave[sl(id, m)] = v;  // natural row n2 + R2 (m % NB) of block m / NB, in place
            }
          });
    }
    if constexpr (DIR > 0 && G > 1) {
      send_block(wave, rank, 2, 1, 0);
      Base::exchange_wait(wave, 0);
    } else {
      __syncthreads();
    }
  }

  // ---- column contiguous (spectral side) --------------------------------
  template <bool FROM_SMEM, bool FWD, bool INV, bool WB = false, class Load, class Op>
  __device__ static void col_contig(float2* wave, const float2* twC, int rank, const Load& load, const Op& op) {
    const int warp = threadIdx.x >> 5;
    TcMat<MODE> M;
    load_mat<R2>(M);
    auto sl = [&](int id, int e) {
      const int k1 = id / ROWS, cc = id % ROWS;
      return cslot(rank, k1 / NB, R2 * (k1 % NB) + e, cc);
    };
    auto pu_pv = [&](int id, int e, int& pu, int& pv) {
      const int k1 = id / ROWS, cc = id % ROWS;
      pu = R2 * k1 + e;
      pv = rank * ROWS + cc;
    };
#pragma unroll 1
    for (int q = warp; q < TC / 8; q += WARPS) {
      const int task0 = 8 * q;
      if constexpr (FWD) {
        tc_dft8<MODE, R2, false>(
            M, task0, [&](int id, int e) { return wave[sl(id, e)]; },
            [&](int id, int m, float2 v) {
              if constexpr (INV) {
                wave[sl(id, m)] = v;
              } else {
                int pu, pv;
                pu_pv(id, m, pu, pv);
                if (chk(pu >= 0 && pu < N && pv >= 0 && pv < N, kChkWindow)) op(pu, pv, v);
                if constexpr (WB) wave[sl(id, m)] = v;
              }
            });
        if constexpr (INV) __syncwarp();
      }
      if constexpr (INV) {
        tc_dft8<MODE, R2, true>(
            M, task0,
            [&](int id, int e) {
              int pu, pv;
              pu_pv(id, e, pu, pv);
              float2 v = make_float2(0.f, 0.f);
              if (!chk(pu >= 0 && pu < N && pv >= 0 && pv < N, kChkWindow)) return v;
              if constexpr (FWD || FROM_SMEM) v = wave[sl(id, e)];
              else v = load(pu, pv);
              op(pu, pv, v);
              return v;
            },
            [&](int id, int m, float2 v) {
              const int k1 = id / ROWS;
              wave[sl(id, m)] = m ? cmulc(v, twC[m * R1 + k1]) : v;
            });
      }
    }
  }

  __device__ static void inverse_tail(float2* wave, const float2* twS, const float2* twC, int rank) {
    col_strided<+1>(wave, twS, rank);
    row_contig<+1>(wave, twC, rank);
  }
  __device__ static void forward_mid(float2* wave, const float2* twS, const float2* twC, int rank) {
    row_contig<-1>(wave, twC, rank);
    col_strided<-1>(wave, twS, rank);
  }
};

}  // namespace ptycho
