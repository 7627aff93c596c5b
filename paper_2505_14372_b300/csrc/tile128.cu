// Window 128x128: 1-CTA cluster per wavefield, 128 = 8 x 16, 1024 threads
// (every thread one contiguous-stage task and two strided ones; measured
// against 512 threads: 356 -> 341 us per tile launch of the 4-mode,
// 256-position step, despite the spills that 64 registers per thread cost).
#include "engine_impl.cuh"

namespace ptycho {
using Tile128 = Tile<128, 1, 16, 1024, 1>;
const EngineOps* engine_128() { return Engine<Tile128>::ops(); }
}  // namespace ptycho
