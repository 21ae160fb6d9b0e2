// Engine instantiation for the float cycle.
#include "engine.cuh"

namespace wadr {
EngineBase* make_engine_f32() { return new Engine<float>(); }
}  // namespace wadr
