// fp32 instantiation of the FFT-LB engine (FFTs and pointwise work in fp32,
// conservation sums in fp64).
#include "engine_impl.cuh"

namespace fftlb {
Engine *make_engine_f32() { return new EngineT<float>(); }
}  // namespace fftlb
