// Choice of form and precision when the caller leaves them to the library (M2L_FORM_AUTO /
// M2L_PREC_AUTO), per (p, n_rhs, target tolerance).
#include "internal.h"

namespace m2l {

int resolve_form(const m2l_plan_t *pl, int R, int *form, int *precision) {
    (void)R;
    int f = pl->form, pr = pl->precision;
    if (pr == M2L_PREC_AUTO) pr = pl->target_tol < 1e-6 ? M2L_PREC_FP64 : M2L_PREC_FP32;
    if (f == M2L_FORM_AUTO) f = M2L_FORM_BLAS;
    *form = f;
    *precision = pr;
    return M2L_OK;
}

}  // namespace m2l
