// Access to a lattice context's layout and clock for the surrogate window
// (lbm_surrogate_advance in lbm_fno.cu), without the step kernels' headers.
#pragma once
#include "../../include/lbm.h"

namespace lbm {
// lattice id, nodes per axis, current time, and whether the context is
// initialised without a sticky error
void ctx_window_info(const lbm_ctx *c, int *lattice, int n[3], long long *t, int *ready);
// the clock after a re-initialisation from fields that stand for time t
void ctx_set_time(lbm_ctx *c, long long t);
// lbm_init from device fields already checked on the device (every alpha_g in
// [0, 1], their sum alpha_sum): no host copy of alpha_g
int ctx_init_device(lbm_ctx *c, const double *alpha_g, const double *u_g, const double *u_l, const double *p_k,
                    double alpha_sum);
// record an error message on the context (lbm_last_error)
int ctx_error(lbm_ctx *c, int code, const char *msg);
}  // namespace lbm
