// Window 256x256: 4-CTA cluster per wavefield, 256 = 16 x 16, 512 threads.
#include "engine_impl.cuh"

namespace ptycho {
using Tile256 = Tile<256, 4, 16, 512, 1>;
const EngineOps* engine_256() { return Engine<Tile256>::ops(); }
}  // namespace ptycho
