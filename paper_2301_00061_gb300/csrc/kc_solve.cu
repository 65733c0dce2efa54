// kc_solve.cu -- placeholder entry points, replaced by the tightening and solver implementation.
#include "kc_internal.cuh"
using namespace kc;
extern "C" {
kc_status kc_tighten(kc_ctx *c, const void *, const void *, int32_t, double, const int64_t *, int32_t, void *,
                     void *, int64_t *, int64_t *, double *, int8_t *)
{
    return set_err(c, KC_EINTERNAL, "kc_tighten: not available in this build");
}
kc_status kc_sample_reduction(kc_ctx *c, const void *, const void *, int32_t, const int64_t *, int32_t, double,
                              double, uint8_t *, int64_t *)
{
    return set_err(c, KC_EINTERNAL, "kc_sample_reduction: not available in this build");
}
void kc_solve_defaults(kc_solve_opts *o)
{
    *o = kc_solve_opts{};
    o->tol = 1e-12;
    o->ball_cap = 50;
    o->i_sr = 1;
    o->use_bt = 1;
    o->use_graph = 1;
}
kc_status kc_solve(kc_ctx *c, double, const kc_solve_opts *, kc_result *)
{
    return set_err(c, KC_EINTERNAL, "kc_solve: not available in this build");
}
}
