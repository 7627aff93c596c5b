// Window 192x192: 2-CTA cluster per wavefield, 192 = 12 x 16, 384 threads
// (every stage then gives each thread a whole number of tasks: 4 strided,
// 3 contiguous).
#include "engine_impl.cuh"

namespace ptycho {
using Tile192 = Tile<192, 2, 16, 384, 1>;
const EngineOps* engine_192() { return Engine<Tile192>::ops(); }
}  // namespace ptycho
