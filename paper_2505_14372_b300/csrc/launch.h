// Launch descriptors shared by the host runtime and the kernels.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace ptycho {

constexpr int kMaxDesc = 16;           // problems per batched launch
constexpr unsigned PTYCHO_STATUS_OUT_OF_BOUNDS = 1u;
constexpr int kModelEpie = 3;                      // noise-model id of the ePIE modulus update

// Kernel variants of the forward / adjoint kernels: the storage format of
// the entry-wave copies (FP32, binary16, bfloat16) and the ePIE normalisers
// are compile-time properties of their real-space stages.
// LSQML (§3.3.2) runs two passes: kVarLsqDir accumulates the update
// directions (the plain adjoint chain from the modulus-update seed) and the
// group's illumination; kVarLsqStep recomputes the chain and reduces the
// per-position least-squares step sizes, then scatters the step-weighted
// illumination.
// kVarDet (position-major kernel only) keeps each position's object- and
// probe-gradient contributions apart (ProblemDesc::det_gO / det_gP) instead
// of adding them with atomics, for fixed-order sums afterwards.
enum Variant { kVarF32 = 0, kVarF16 = 1, kVarBF16 = 2, kVarEpie = 3, kVarLsqDir = 4, kVarLsqStep = 5, kVarDet = 6 };

// One problem (dataset) inside a launch.  All pointers are device pointers.
struct ProblemDesc {
  const float2* O;      // [S][H][W] object slices
  const float2* Phat;   // [K][NP] probe spectra, spectral slot order
  const float* pos;     // [*][2] scan positions (y, x), window top-left
  const int* idx;       // [B] minibatch -> position index (null: identity)
  const float2* Hc;     // [S-1][N] separable Fresnel chirp per gap, slot order
  float2* A;            // [B][K][NP] far field F(phi), slot order
  const float* w;       // [B][NP] 2 l'(I) / NP, slot order (adjoint)
  char* waves;          // STORE: [B][K][S][NP] entry waves (natural order, the variant's format)
  float2* gO;           // [S][H][W] object gradient (accumulated)
  float2* gPhat;        // [K][NP] probe spectrum gradient (accumulated)
  double* gpos;         // [B][2] scan-position gradient (accumulated), or null
  int S, K, H, W, B;
  int npos;             // rows of pos (and of the pattern array) idx may select
  int blT;              // band limit keeps f_u^2 + f_v^2 <= blT; < 0: off
  int item0;            // first global item (position-major kernel: position) of this problem
  // position-major loss + adjoint: measured patterns [npos][NP] (natural
  // order), loss per position [B] (zeroed per launch) and the noise model
  const float* Iexp;
  double* lpart;
  int model;
  float eps, c;
  // ePIE (null for the gradient): max |O_s|^2 per slice [S] and max |psi_s|^2
  // per item and slice [B][K][S], both as float bits (atomicMax)
  const unsigned* omax;
  unsigned* wmax;
  // LSQML (null otherwise): illumination [S][H][W] (direction pass), object
  // direction [S][H][W] and probe-direction spectra [K][NP] (slot order),
  // step-size sums per position and slice [B][S] and per position [B], and
  // the step-weighted illumination [S][H][W] (step pass)
  float* lsq_il;
  const float2* lsq_dO;
  const float2* lsq_dPhat;
  double* lsq_num;
  double* lsq_den;
  double* lsq_numP;
  double* lsq_denP;
  float* lsq_aw;
  // deterministic reduction (kVarDet): per-position object-gradient patches
  // [B][S][NP] (natural order, summed over the modes in mode order) and
  // probe-spectrum gradients [B][K][NP] (slot order)
  float2* det_gO;
  float2* det_gP;
};

struct LaunchArgs {
  ProblemDesc d[kMaxDesc];
  int nd;
  int total;                // items over all problems
  unsigned* status;         // device status word (PTYCHO_STATUS_*)
  char* slots;              // recompute scratch, one slot per cluster
  long long slot_stride;    // bytes per slot
  // item-major kernels, one-problem launches: processing order of the
  // positions ([B], a permutation; the items of position order[p] are taken
  // at p K .. p K + K - 1), or null for item order
  const int* order;
};

// Extra arguments of the position-major loss + adjoint kernel: one cluster
// per scan position runs the forward pass of every mode, the noise model on
// the mode sum, then the backward pass of every mode.  Per-cluster scratch:
// far fields and intensity / seed weights (and K entry-wave sets in the slot).
// The positions of a launch are those of all its problems in order
// (LaunchArgs::total of them, ProblemDesc::item0 the first of each).
struct PosArgs {
  float2* Abuf;        // [clusters][astride] far fields F(phi) of the modes, slot order
  float* Ibuf;         // [clusters][NP] mode-summed intensity, then 2 l'(I) / NP
  long long astride;   // float2 per cluster in Abuf (>= K NP of every problem)
  float gamma;         // LSQML step-size regulariser
  // processing order [total]: a permutation of the launch's positions,
  // taken in this order, or null for 0, 1, ...; outputs stay indexed by
  // position
  const int* order;
  // work queue of the launch: [0] next entry of the order to claim, [1]
  // clusters done.  Both zero when a launch starts; the last cluster to
  // finish sets them back to zero.
  unsigned* queue;
};

// Fused end of a gradient step for single-CTA tiles (N <= 128): probe
// gradient g_P_k = F^-1 g_P^_k (one block per mode), the complex Adam updates
// of the probe (from the block's shared memory) and of the object, the FP64
// |g|^2 block partials, and, in the last block to finish, the final loss and
// gradient-norm sums.  It also clears what the next step accumulates into
// (g_P^, g_O and the per-position loss partials), so that step needs no
// memsets.
struct TailArgs {
  float2* gPhat;        // [K][NP] probe spectrum gradient, slot order (read, then zeroed)
  float2* P;            // [K][NP] probe (updated when update_probe)
  float2* mP;
  float* vP;
  float2* O;            // [nO] object (updated)
  float2* mO;
  float* vO;
  float2* gO;           // [nO] object gradient (read, then zeroed)
  long long nO;
  int K, update_probe;
  float lrO, lrP, b1, b2, eps, bc1, bc2;
  const float* bcd;     // bias corrections in device memory (step counter on the device), or null
  double* lossp;        // [nl] loss partials (summed, then [0, nz) zeroed)
  int nl, nz;
  double* normp;        // [gridDim.x] FP64 |g|^2 partial of each block
  double* stats;        // out: [0] loss, [1] gradient norm
  unsigned* counter;    // blocks done (0 between launches; reset by the last block)
};

}  // namespace ptycho
