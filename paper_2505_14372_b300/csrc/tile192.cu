// Window 192x192: 2-CTA cluster per wavefield, 192 = 12 x 16, 576 threads.
#include "engine_impl.cuh"

namespace ptycho {
using Tile192 = Tile<192, 2, 16, 576, 1>;
const EngineOps* engine_192() { return Engine<Tile192>::ops(); }
}  // namespace ptycho
