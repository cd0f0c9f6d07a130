// The instrumented build of the wavefront decoder (decode_kernel with
// PROF = true), in a compilation unit of its own.
#include "nlc_decode_kernel.cuh"

namespace nlc {

const void* decode_fn_prof(int prec, bool win) {
  if (win) return (const void*)decode_kernel<PREC_BF16, false, true, true>;
  return prec == PREC_BF16 ? (const void*)decode_kernel<PREC_BF16, false, false, true>
                           : (const void*)decode_kernel<PREC_FP32, false, false, true>;
}

}  // namespace nlc
