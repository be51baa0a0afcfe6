// Device-resident state of one forward step or one backward step.
#pragma once

#include <cstdint>

namespace pd {

constexpr int kMaxHistory = 16;

struct IterState {
  // forward: objective g; backward: quadratic s(z) = z^T H z / 2 - gbar^T z
  double alpha;          // step length of the current trial
  double slope;          // d . grad at the accepted point
  double g_acc;          // objective at the accepted point (forward)
  double gn2_acc;        // |grad|^2 at the accepted point
  double ref2;           // convergence reference squared
  double refM2;          // forward: |M y / h^2|^2 on the free DoFs
  double g_t, gn2_t, gd_t, dHd;
  double tol2;
  double c1;
  double noise;          // relative objective noise accepted by the Armijo test
  double rho[kMaxHistory], al[kMaxHistory], cf[kMaxHistory];
  double sg[kMaxHistory];                // s_i . g at the current gradient
  double SY[kMaxHistory][kMaxHistory];   // s_i . y_j of the stored pairs (ring slots)
  double aux;            // scalar accumulator (friction coefficient gradient)
  int m;                 // history capacity
  int head, count;
  int pslot, push;
  int iters, evals, ls_tries, ls_total, ls_max, max_iter;
  int accepted, converged, hit_max, force_accept, fp64_checked;
  int pending;           // backward: a step (alpha, d, Hd) waits to be applied
  int svd_cached;        // backward: the step's FP32 point SVDs are in the mesh's cache
  int status;            // DEV_ERR_* bits
};

}  // namespace pd
