// fp64 instantiation of the FFT-LB engine.
#include "engine_impl.cuh"

namespace fftlb {
Engine *make_engine_f64() { return new EngineT<double>(); }
}  // namespace fftlb
