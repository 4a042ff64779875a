// fp32 instantiation of the FFT-LB engine with the split-BF16 tensor-core
// first radix-16 passes (precision 32 | FFTLB_BF16SPLIT).
#include "engine_impl.cuh"

namespace fftlb {
Engine *make_engine_f32_split() { return new EngineT<float, true>(); }
}  // namespace fftlb
