// Entry points of libse under the names of the problem statement (Sec. 2: the potential of
// N point sources in a D-periodic box; Alg. 1 input): se_plan, the plan constructor, and
// se_eval_batch, the evaluation of many independent configurations in one call. Both are
// host code over the primary entry points of se_core.cu.
#include "../../include/se.h"

extern "C" se_status se_plan(se_plan_h* out, int periodicity, const double box[3], double xi, double rc,
                             const int M[3], int P, int window, const se_opts* opts) {
  return se_plan_create(out, periodicity, box, xi, rc, M, P, window, opts);
}

extern "C" se_status se_eval_batch(const se_plan_h* plans, int n_cfg, const int* kernel_mask,
                                   const long long* n_src, const double* const* src,
                                   const void* const* strengths, const int* n_rhs, void* const* u) {
  if (n_cfg < 1 || !plans || !kernel_mask || !n_src || !src || !strengths || !n_rhs || !u) return SE_ERR_ARG;
  for (int i = 0; i < n_cfg; ++i)
    if (!plans[i]) return SE_ERR_ARG;
  for (int i = 0; i < n_cfg; ++i) {
    const se_status s = se_eval(plans[i], kernel_mask[i], n_src[i], src[i], strengths[i], n_rhs[i], 0, nullptr, u[i]);
    if (s != SE_OK) return s;
  }
  return SE_OK;
}
