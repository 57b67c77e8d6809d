// The double operator kernels (see operator_kernels.cuh), compiled apart from
// the other precisions so the library's translation units build in parallel.
#include "operator_kernels.cuh"

namespace mm {

const OpImpl& op_impl_f64() {
  static const OpImpl impl = make_impl<double>();
  return impl;
}

}  // namespace mm
