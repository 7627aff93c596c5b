// FP64 reductions and the complex Adam update (arXiv 2505.14372 §3.2).
#include <algorithm>
#include <atomic>

#include "elementwise.cuh"
#include "engine.h"
#include "ptycho.h"

namespace ptycho {

namespace {
std::atomic<unsigned long long> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// Block partial sums of |g|^2 over a complex array (FP64).
__global__ void __launch_bounds__(kRedThreads) k_sumsq(const float2* __restrict__ g, long long n,
                                                       double* __restrict__ partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float2 v = __ldg(g + e);
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// out[0] = sum of partials[0..n0), out[1] = sqrt(sum of partials[n0..n0+n1))
// (fixed summation order: deterministic).
__global__ void __launch_bounds__(kRedThreads) k_finalize(const double* __restrict__ partials, int n0, int n1,
                                                          double* __restrict__ out, int sqrt_second) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n0; i += blockDim.x) a += partials[i];
  for (int i = threadIdx.x; i < n1; i += blockDim.x) b += partials[n0 + i];
  const double ta = block_sum(a, sh);
  const double tb = block_sum(b, sh);
  if (threadIdx.x == 0) {
    out[0] = ta;
    if (n1 > 0) out[1] = sqrt_second ? sqrt(tb) : tb;
  }
}

// Complex Adam: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2)|g|^2;
// z <- z - lr (m bc1) / (sqrt(v bc2) + eps), bc = 1/(1 - beta^t).
// With `partials` the block also writes its FP64 partial of |g|^2 (the same
// elements per block and order as k_sumsq on the same grid).
__global__ void __launch_bounds__(kRedThreads) k_adam(float2* __restrict__ z, float2* __restrict__ m,
                                                      float* __restrict__ v, const float2* __restrict__ g,
                                                      long long n, float lr, float b1, float b2, float eps,
                                                      float bc1, float bc2, const float* __restrict__ bcd,
                                                      double* __restrict__ partials) {
  __shared__ double sh[32];
  if (bcd) {  // bias corrections of a step count kept in device memory
    bc1 = bcd[0];
    bc2 = bcd[1];
  }
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float2 gg = g[e];
    if (partials) acc += (double)gg.x * gg.x + (double)gg.y * gg.y;
    adam_elem(z, m, v, e, gg, lr, b1, b2, eps, bc1, bc2);
  }
  if (partials) {
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}


// Cost regularisers (arXiv 2505.14372 §3.4) on the complex transmission and
// the probe: adds their gradients (dL/dRe z + i dL/dIm z) to gO / gP and
// writes block partial sums of their value.  Object elements [0, nO), probe
// elements [nO, nO + nP).  Object L2 penalises the distance to vacuum
// (O = 1); Tikhonov (squared) and TV (smoothed modulus
// sqrt(|d|^2 + eta^2) - eta) terms use forward differences d inside each
// slice (y, x) and across layers (s).
__global__ void __launch_bounds__(kRedThreads) k_regularize(const float2* __restrict__ O, float2* __restrict__ gO,
                                                            int S, int H, int W, const float2* __restrict__ P,
                                                            float2* __restrict__ gP, long long nP, float l2,
                                                            float tik, float lay, float l2p, float tv,
                                                            float tvl, float eta, double* __restrict__ partials) {
  __shared__ double sh[32];
  const long long HW = (long long)H * W, nO = (long long)S * HW;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nO + nP;
       e += (long long)gridDim.x * blockDim.x) {
    if (e >= nO) {
      const long long i = e - nO;
      const float2 p = P[i];
      acc += (double)l2p * cabs2(p);
      float2 g = gP[i];
      g.x += 2.f * l2p * p.x;
      g.y += 2.f * l2p * p.y;
      gP[i] = g;
      continue;
    }
    const int s = (int)(e / HW);
    const long long r = e - (long long)s * HW;
    const int y = (int)(r / W), x = (int)(r - (long long)y * W);
    const float2 o = O[e];
    float gx = 0.f, gy = 0.f;
    float val = 0.f;
    if (l2 != 0.f) {
      const float dx_ = o.x - 1.f, dy_ = o.y;
      val += l2 * (dx_ * dx_ + dy_ * dy_);
      gx += 2.f * l2 * dx_;
      gy += 2.f * l2 * dy_;
    }
    auto edge = [&](float lam, long long nb, bool fwd) {
      const float2 q = O[nb];
      const float dx_ = o.x - q.x, dy_ = o.y - q.y;
      if (fwd) val += lam * (dx_ * dx_ + dy_ * dy_);  // each difference counted once
      gx += 2.f * lam * dx_;
      gy += 2.f * lam * dy_;
    };
    if (tik != 0.f) {
      if (y + 1 < H) edge(tik, e + W, true);
      if (y > 0) edge(tik, e - W, false);
      if (x + 1 < W) edge(tik, e + 1, true);
      if (x > 0) edge(tik, e - 1, false);
    }
    if (lay != 0.f) {
      if (s + 1 < S) edge(lay, e + HW, true);
      if (s > 0) edge(lay, e - HW, false);
    }
    auto tv_edge = [&](float lam, long long nb, bool fwd) {
      const float2 q = O[nb];
      const float dx_ = o.x - q.x, dy_ = o.y - q.y;
      const float r = sqrtf(dx_ * dx_ + dy_ * dy_ + eta * eta);
      if (fwd) val += lam * (r - eta);
      const float f = lam / r;
      gx += f * dx_;
      gy += f * dy_;
    };
    if (tv != 0.f) {
      if (y + 1 < H) tv_edge(tv, e + W, true);
      if (y > 0) tv_edge(tv, e - W, false);
      if (x + 1 < W) tv_edge(tv, e + 1, true);
      if (x > 0) tv_edge(tv, e - 1, false);
    }
    if (tvl != 0.f) {
      if (s + 1 < S) tv_edge(tvl, e + HW, true);
      if (s > 0) tv_edge(tvl, e - HW, false);
    }
    float2 g = gO[e];
    g.x += gx;
    g.y += gy;
    gO[e] = g;
    acc += (double)val;
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

cudaError_t launch_regularize(const float2* O, float2* gO, int S, int H, int W, const float2* P, float2* gP,
                              long long nP, float l2, float tik, float lay, float l2p, float tv, float tvl,
                              float eta, double* partials, int nblocks, cudaStream_t s) {
  count_launch();
  k_regularize<<<nblocks, kRedThreads, 0, s>>>(O, gO, S, H, W, P, gP, nP, l2, tik, lay, l2p, tv, tvl, eta, partials);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const float2* g, long long n, double* partials, int nblocks, cudaStream_t s) {
  count_launch();
  k_sumsq<<<nblocks, kRedThreads, 0, s>>>(g, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int n0, int n1, double* out, int sqrt_second,
                            cudaStream_t s) {
  count_launch();
  k_finalize<<<1, kRedThreads, 0, s>>>(partials, n0, n1, out, sqrt_second);
  return cudaGetLastError();
}

cudaError_t launch_adam(float2* z, float2* m, float* v, const float2* g, long long n, float lr, float b1,
                        float b2, float eps, float bc1, float bc2, cudaStream_t s, const float* bcd,
                        double* norm_partials) {
  if (n <= 0 && !norm_partials) return cudaSuccess;
  const int blocks = norm_partials ? kNormBlocks : (int)std::min<long long>((n + 255) / 256, 148LL * 16);
  count_launch();
  k_adam<<<blocks, kRedThreads, 0, s>>>(z, m, v, g, n, lr, b1, b2, eps, bc1, bc2, bcd, norm_partials);
  return cudaGetLastError();
}

// Adam step count in device memory (one thread): t <- t + 1 and the bias
// corrections 1 / (1 - beta^t) of the new count, in FP64, into bc[2].
__global__ void k_adam_count(long long* t, float b1, float b2, float* bc) {
  const long long t1 = *t + 1;
  bc[0] = (float)(1.0 / (1.0 - pow((double)b1, (double)t1)));
  bc[1] = (float)(1.0 / (1.0 - pow((double)b2, (double)t1)));
  *t = t1;
}

// Processing order of a position-major launch.  The clusters running at one
// time take consecutive entries of the order, so sorting the positions along
// a Hilbert curve of their window origins makes those clusters read
// neighbouring, overlapping object patches, which then serve each other
// from L2.  Rank sort (stable: ties by position index), one thread per
// position against tiles of keys in shared memory.
__device__ unsigned long long locality_key(const LaunchArgs& L, int it) {
  int d = 0;
  while (d + 1 < L.nd && it >= L.d[d + 1].item0) ++d;
  const ProblemDesc& D = L.d[d];
  const int j = it - D.item0;
  const int jj = D.idx ? D.idx[j] : j;
  unsigned y = 0, x = 0;
  if (jj >= 0 && jj < D.npos) {  // out-of-range positions are flagged by the kernel itself
    y = (unsigned)fminf(fmaxf(D.pos[2 * (size_t)jj], 0.f), 65535.f);
    x = (unsigned)fminf(fmaxf(D.pos[2 * (size_t)jj + 1], 0.f), 65535.f);
  }
  // index along a Hilbert curve of order 16 (no jumps between neighbours)
  unsigned h = 0;
  for (unsigned sq = 1u << 15; sq > 0; sq >>= 1) {
    const unsigned ry = (y & sq) ? 1u : 0u, rx = (x & sq) ? 1u : 0u;
    h += sq * sq * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = 0xffffu - x;
        y = 0xffffu - y;
      }
      const unsigned t = x;
      x = y;
      y = t;
    }
  }
  return ((unsigned long long)d << 32) | h;
}
__global__ void __launch_bounds__(kRedThreads) k_locality_order(const __grid_constant__ LaunchArgs L, int* order) {
  __shared__ unsigned long long tile[kRedThreads];
  const int it = blockIdx.x * kRedThreads + threadIdx.x;
  const bool mine = it < L.total;
  const unsigned long long key = mine ? locality_key(L, it) : 0ull;
  int rank = 0;
  for (int base = 0; base < L.total; base += kRedThreads) {
    const int i = base + threadIdx.x;
    tile[threadIdx.x] = i < L.total ? locality_key(L, i) : ~0ull;
    __syncthreads();
    const int n = min(kRedThreads, L.total - base);
    for (int q = 0; q < n; ++q) {
      const unsigned long long kq = tile[q];
      rank += (kq < key || (kq == key && base + q < it)) ? 1 : 0;
    }
    __syncthreads();
  }
  if (mine) order[rank] = it;
}
cudaError_t launch_locality_order(const LaunchArgs& L, int* order, cudaStream_t s) {
  if (L.total <= 0) return cudaSuccess;
  count_launch();
  k_locality_order<<<(L.total + kRedThreads - 1) / kRedThreads, kRedThreads, 0, s>>>(L, order);
  return cudaGetLastError();
}

cudaError_t launch_adam_count(long long* t, float b1, float b2, float* bc, cudaStream_t s) {
  count_launch();
  k_adam_count<<<1, 1, 0, s>>>(t, b1, b2, bc);
  return cudaGetLastError();
}

// max |O_s|^2 of every slice (ePIE object normaliser, §3.3.1) as float
// bits in omax[S] (zeroed by the caller): grid-stride per slice, block max,
// one atomicMax per block.
__global__ void k_slice_absmax(const float2* __restrict__ O, long long per_slice, unsigned* omax) {
  __shared__ float sh[32];
  const int s = blockIdx.y;
  const float2* Os = O + (size_t)s * per_slice;
  float m = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per_slice;
       e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, cabs2(__ldg(Os + e)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = m;
  __syncthreads();
  if (warp == 0) {
    m = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative floats order like their bit patterns
    if (lane == 0) atomicMax(omax + s, __float_as_uint(m));
  }
}

cudaError_t launch_slice_absmax(const float2* O, int S, long long per_slice, unsigned* omax, cudaStream_t s) {
  if (S <= 0 || per_slice <= 0) return cudaSuccess;
  const int bx = (int)std::max<long long>(1, std::min<long long>((per_slice + 255) / 256, (148LL * 8 + S - 1) / S));
  count_launch();
  k_slice_absmax<<<dim3(bx, S), 256, 0, s>>>(O, per_slice, omax);
  return cudaGetLastError();
}

// z += a * g (the ePIE object and probe updates, §3.3.1)
__global__ void k_axpy(float2* __restrict__ z, const float2* __restrict__ g, long long n, float a) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float2 d = __ldg(g + e);
    float2 v = z[e];
    v.x = fmaf(a, d.x, v.x);
    v.y = fmaf(a, d.y, v.y);
    z[e] = v;
  }
}

cudaError_t launch_axpy(float2* z, const float2* g, long long n, float a, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
  count_launch();
  k_axpy<<<blocks, 256, 0, s>>>(z, g, n, a);
  return cudaGetLastError();
}

// LSQML (§3.3.2) helpers.
// Transmission prod_s |O_s|^2 of every position's window, summed into the
// probe frame T[N][N]; with step sums, weighted by the position's probe step
// num[j] / (den[j] + gamma).  Positions outside [0, npos) or the object add
// nothing.
__global__ void k_transmission(const float2* __restrict__ O, int S, int H, int W, int N, const float* __restrict__ pos,
                               const int* __restrict__ idx, int npos, int B, const double* __restrict__ num,
                               const double* __restrict__ den, float gamma, float* __restrict__ T) {
  const long long NP = (long long)N * N, total = (long long)B * NP;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / NP);
    const int p = (int)(e - (long long)j * NP);
    const int jj = idx ? idx[j] : j;
    if (jj < 0 || jj >= npos) continue;
    const double fy = floor((double)pos[2 * (size_t)jj] + 0.5), fx = floor((double)pos[2 * (size_t)jj + 1] + 0.5);
    if (!(fy >= 0.0 && fx >= 0.0 && fy + N <= (double)H && fx + N <= (double)W)) continue;
    const int r = p / N, c = p - r * N;
    const float2* o = O + ((size_t)fy + r) * W + (size_t)fx + c;
    float t = 1.f;
    for (int s = 0; s < S; ++s) t *= cabs2(__ldg(o + (size_t)s * H * W));
    float wgt = 1.f;
    if (num) {
      const double d = den[j] + (double)gamma;
      wgt = d > 0.0 ? (float)(num[j] / d) : 0.f;
    }
    atomicAdd(T + p, wgt * t);
  }
}

// out[e] = num[e] / (den[e % period] + reg), 0 where that is not positive
// (den = den_prev when given)
__global__ void k_divide(const float2* __restrict__ num, const float* __restrict__ den, const float* __restrict__ den_prev,
                         float reg, long long n, long long period, float2* __restrict__ out) {
  const float* d = den_prev ? den_prev : den;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float q = __ldg(d + e % period) + reg;
    const float2 v = __ldg(num + e);
    out[e] = q > 0.f ? make_float2(v.x / q, v.y / q) : make_float2(0.f, 0.f);
  }
}

// z[e] += beta dz[e] aw[e % period] / w[e % period] (unchanged where w = 0)
__global__ void k_weighted_update(float2* __restrict__ z, const float2* __restrict__ dz, const float* __restrict__ aw,
                                  const float* __restrict__ w, float beta, long long n, long long period) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long q = e % period;
    const float ww = __ldg(w + q);
    if (!(ww > 0.f)) continue;
    const float f = beta * __ldg(aw + q) / ww;
    const float2 d = __ldg(dz + e);
    float2 v = z[e];
    v.x = fmaf(f, d.x, v.x);
    v.y = fmaf(f, d.y, v.y);
    z[e] = v;
  }
}

// y[e] += x[e] (float)
__global__ void k_add(float* __restrict__ y, const float* __restrict__ x, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += __ldg(x + e);
}

static int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 148LL * 16)); }

cudaError_t launch_transmission(const float2* O, int S, int H, int W, int N, const float* pos, const int* idx, int npos,
                                int B, const double* num, const double* den, float gamma, float* T, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  count_launch();
  k_transmission<<<grid_for((long long)B * N * N), 256, 0, s>>>(O, S, H, W, N, pos, idx, npos, B, num, den, gamma, T);
  return cudaGetLastError();
}
cudaError_t launch_divide(const float2* num, const float* den, const float* den_prev, float reg, long long n,
                          long long period, float2* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_divide<<<grid_for(n), 256, 0, s>>>(num, den, den_prev, reg, n, period, out);
  return cudaGetLastError();
}
cudaError_t launch_weighted_update(float2* z, const float2* dz, const float* aw, const float* w, float beta, long long n,
                                   long long period, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_weighted_update<<<grid_for(n), 256, 0, s>>>(z, dz, aw, w, beta, n, period);
  return cudaGetLastError();
}
// ---- deterministic gradient sums (geometry flag `deterministic`) ----------
// Object: one thread per object pixel of a 32 x 8 tile of one slice.  The
// group's positions are taken in chunks of kDetChunk in index order; each
// chunk's positions whose window meets the tile are compacted in that order
// (warp ballots, then the warps' offsets), and every thread adds the patch
// values of those that cover its pixel.  The sum therefore runs over the
// positions in index order whatever the launch's processing order was.
// Positions whose window leaves the object (skipped by the tile kernel) are
// skipped here by the same test.
constexpr int kDetTileX = 32, kDetTileY = 8, kDetChunk = 256;
__global__ void __launch_bounds__(kDetChunk) k_det_object_reduce(const float2* __restrict__ patches,
                                                                  const float* __restrict__ pos,
                                                                  const int* __restrict__ idx, int npos, int B, int S,
                                                                  int H, int W, int N, float2* __restrict__ gO) {
  __shared__ int list_j[kDetChunk];
  __shared__ int list_y[kDetChunk];
  __shared__ int list_x[kDetChunk];
  __shared__ int warp_n[kDetChunk / 32];
  __shared__ int total;
  const int tx = (W + kDetTileX - 1) / kDetTileX, ty = (H + kDetTileY - 1) / kDetTileY;
  const int s = blockIdx.x / (tx * ty);
  const int t = blockIdx.x % (tx * ty);
  const int y0 = (t / tx) * kDetTileY, x0 = (t % tx) * kDetTileX;
  const int y = y0 + threadIdx.x / kDetTileX, x = x0 + threadIdx.x % kDetTileX;
  const bool mine = y < H && x < W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t NP = (size_t)N * N;
  float2 acc = make_float2(0.f, 0.f);
  for (int c0 = 0; c0 < B; c0 += kDetChunk) {
    const int j = c0 + (int)threadIdx.x;
    bool hit = false;
    int ny = 0, nx = 0;
    if (j < B) {
      const int jj = idx ? idx[j] : j;
      if (jj >= 0 && jj < npos) {
        const double fy = floor((double)pos[2 * (size_t)jj] + 0.5), fx = floor((double)pos[2 * (size_t)jj + 1] + 0.5);
        const bool ok = fy >= 0.0 && fx >= 0.0 && fy + N <= (double)H && fx + N <= (double)W;
        ny = (int)fy;
        nx = (int)fx;
        hit = ok && ny < y0 + kDetTileY && ny + N > y0 && nx < x0 + kDetTileX && nx + N > x0;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) warp_n[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
      int a = 0;
      for (int w = 0; w < kDetChunk / 32; ++w) {
        const int n = warp_n[w];
        warp_n[w] = a;
        a += n;
      }
      total = a;
    }
    __syncthreads();
    if (hit) {
      const int o = warp_n[warp] + __popc(m & ((1u << lane) - 1u));
      list_j[o] = j;
      list_y[o] = ny;
      list_x[o] = nx;
    }
    __syncthreads();
    if (mine) {
      for (int i = 0; i < total; ++i) {
        const int dy = y - list_y[i], dx = x - list_x[i];
        if (dy >= 0 && dy < N && dx >= 0 && dx < N)
          acc = cadd(acc, patches[((size_t)list_j[i] * S + s) * NP + (size_t)dy * N + dx]);
      }
    }
    __syncthreads();
  }
  if (mine) {
    float2* g = gO + ((size_t)s * H + y) * W + x;
    *g = cadd(*g, acc);
  }
}

// Probe spectra: gPhat[k][p] += sum over positions j in index order of
// pgrad[j][k][p].
__global__ void __launch_bounds__(256) k_det_probe_reduce(const float2* __restrict__ pgrad, int B, long long KNP,
                                                          float2* __restrict__ gPhat) {
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < KNP; e += (long long)gridDim.x * 256) {
    float2 a = make_float2(0.f, 0.f);
    for (int j = 0; j < B; ++j) a = cadd(a, pgrad[(size_t)j * KNP + e]);
    gPhat[e] = cadd(gPhat[e], a);
  }
}

cudaError_t launch_det_reduce(const float2* patches, const float2* pgrad, const float* pos, const int* idx, int npos,
                              int B, int S, int K, int H, int W, int N, float2* gO, float2* gPhat, cudaStream_t s) {
  const long long tiles = (long long)((W + kDetTileX - 1) / kDetTileX) * ((H + kDetTileY - 1) / kDetTileY) * S;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  count_launch();
  k_det_object_reduce<<<(unsigned)tiles, kDetChunk, 0, s>>>(patches, pos, idx, npos, B, S, H, W, N, gO);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long KNP = (long long)K * N * N;
  count_launch();
  k_det_probe_reduce<<<(unsigned)std::min<long long>((KNP + 255) / 256, 148LL * 8), 256, 0, s>>>(pgrad, B, KNP, gPhat);
  return cudaGetLastError();
}

cudaError_t launch_add(float* y, const float* x, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_add<<<grid_for(n), 256, 0, s>>>(y, x, n);
  return cudaGetLastError();
}

}  // namespace ptycho

extern "C" uint64_t ptycho_kernels_launched(void) { return ptycho::launches_so_far(); }
