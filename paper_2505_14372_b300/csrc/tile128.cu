// Window 128x128: 1-CTA cluster per wavefield, 128 = 8 x 16, 512 threads.
#include "engine_impl.cuh"

namespace ptycho {
using Tile128 = Tile<128, 1, 16, 512, 1>;
const EngineOps* engine_128() { return Engine<Tile128>::ops(); }
}  // namespace ptycho
