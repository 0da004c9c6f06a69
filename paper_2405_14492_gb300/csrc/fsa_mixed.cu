// Mixed-precision form (placeholder until the tensor-core path lands).
#include "fsa_solver.cuh"

namespace fsa {

void build_operator_mixed(Handle& H, const fsa_theta& th) {
  (void)H;
  (void)th;
  throw Error{FSA_ERR_UNSUPPORTED, "mixed precision not built"};
}

LoglikResult run_loglik_grad_mixed(Handle& H, const fsa_theta& th, const fsa_opts& o) {
  (void)H;
  (void)th;
  (void)o;
  throw Error{FSA_ERR_UNSUPPORTED, "mixed precision not built"};
}

}  // namespace fsa
