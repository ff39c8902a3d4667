// pd_tc.cu -- tensor-core (tcgen05) evaluation of the objective and gradient.
#include "pd_internal.h"

namespace pd {

int eval_tc(const EvalCall& c, cudaStream_t st) {
  (void)c;
  (void)st;
  return PD_ENOTSUP;
}

}  // namespace pd
