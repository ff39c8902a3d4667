// pd_simt_f32_2d.cu -- instantiations of the CUDA-core evaluation for
// float arithmetic on 2-D pixel sets (one translation unit per
// precision and dimension so that the build compiles them in parallel).
#include "pd_simt_kernels.cuh"

namespace pd {

int eval_simt_f32_2d(const EvalCall& c, cudaStream_t st) {
  switch (c.d) {
    case 1: return eval_simt_dd<float, 2, 1>(c, st);
    case 2: return eval_simt_dd<float, 2, 2>(c, st);
    case 3: return eval_simt_dd<float, 2, 3>(c, st);
    case 4: return eval_simt_dd<float, 2, 4>(c, st);
    case 5: return eval_simt_dd<float, 2, 5>(c, st);
    case 6: return eval_simt_dd<float, 2, 6>(c, st);
    case 7: return eval_simt_dd<float, 2, 7>(c, st);
    default: return PD_ENOTSUP;
  }
}

}  // namespace pd
