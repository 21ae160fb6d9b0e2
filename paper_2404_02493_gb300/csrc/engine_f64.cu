// Engine instantiation for the double cycle.
#include "engine.cuh"

namespace wadr {
EngineBase* make_engine_f64() { return new Engine<double>(); }
}  // namespace wadr
