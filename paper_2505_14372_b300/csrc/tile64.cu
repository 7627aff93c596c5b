// Window 64x64: 1-CTA cluster per wavefield, 64 = 4 x 16, 256 threads.
#include "engine_impl.cuh"

namespace ptycho {
using Tile64 = Tile<64, 1, 16, 256, 3>;
const EngineOps* engine_64() { return Engine<Tile64>::ops(); }
}  // namespace ptycho
