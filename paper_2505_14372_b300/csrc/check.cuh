// Index checks of the checked build (compiled with PTYCHO_CHECKED=1 into
// libptycho_checked.so; the normal build compiles them away).
//
// Every shared-memory access of the tile stages goes through the slot
// function, and every global access of a stage's pointwise operations is
// made at window coordinates (row and column, or spectral slots pu and pv)
// relative to per-item base pointers, which are formed from the item's
// position, mode and slice.  The checks sit at those three places: a slot
// index inside the CTA's wavefield, window coordinates inside [0, N), and
// item indices inside their problem.  A failed check records its bit in a
// device word of the tile's translation unit (read and cleared by
// ptycho_check, which then reports PTYCHO_ECHECK) and the access is
// skipped or redirected to slot 0: nothing traps and nothing reads or
// writes outside its buffer.
#pragma once

#ifndef PTYCHO_CHECKED
#define PTYCHO_CHECKED 0
#endif

namespace ptycho {

constexpr unsigned kChkSmem = 1u;    // shared-memory slot outside the wavefield
constexpr unsigned kChkWindow = 2u;  // window coordinate outside [0, N)
constexpr unsigned kChkItem = 4u;    // position / mode / slot index outside its problem

#if PTYCHO_CHECKED
static __device__ unsigned g_check_bits;
__device__ __forceinline__ bool chk(bool ok, unsigned bit) {
  if (!ok) atomicOr(&g_check_bits, bit);
  return ok;
}
#else
__device__ __forceinline__ bool chk(bool, unsigned) { return true; }
#endif

}  // namespace ptycho
