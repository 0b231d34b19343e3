// Per-instance FP64 scalars of the adjoint sweep (the cavity amplitude, its
// cotangent chain, the objective and the parameter gradients), kept on the
// device so that the backward steps run without host round trips.
#pragma once

#include "common.cuh"

namespace mq {

struct AdjScalars {
    double a0_re, a0_im;          // alpha at the start of the step being reversed
    double as_re[4], as_im[4];    // stage amplitudes
    double ka_re[4], ka_im[4];    // stage derivatives d alpha/dt
    double X[4];                  // stage coupling sums (with V_c)
    double la_re, la_im;          // cotangent of alpha after the step
    double lp_re, lp_im;          // the same, kept for the stage cotangents
    double nl_re, nl_im;          // cotangent of alpha before the step (accumulating)
    double lk_re, lk_im;          // cotangent of the current stage's d alpha/dt
    double J;                     // window part of the objective
    double grad[6];               // dJ/d(B_ext x, y, z; eta; omega_c; kappa)
};

}  // namespace mq
