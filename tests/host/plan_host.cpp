// Host build of the step plan and slot layout (peps_plan.h) for CPU tests:
// the bond dimensions of every absorption step and the workspace capacities
// the kernels index with.
#include <cstdint>
#include "peps_plan.h"

extern "C" {

// steps of (L, D, Dc): six int16 arrays [L-1][L] (ia, ip, ib, r, oa, ob) and
// caps = {site_cap, env_cap, big_cap, mat_cap, env2_cap, slot_elems,
// slot_doubles} of the full layout
int h_plan(int L, int D, int Dc, int16_t* ia, int16_t* ip, int16_t* ib, int16_t* r,
           int16_t* oa, int16_t* ob, int64_t* caps) {
  if (L < 2 || L > PEPS_MAXL) return -1;
  PepsPlan P;
  PepsStep steps[PEPS_MAXL];
  peps_plan_steps(L, D, Dc, 1.0, 0.5, &P, steps);
  peps_plan_layout(&P, false);
  for (int t = 0; t < L - 1; ++t)
    for (int j = 0; j < L; ++j) {
      const int o = t * L + j;
      ia[o] = steps[t].ia[j]; ip[o] = steps[t].ip[j]; ib[o] = steps[t].ib[j];
      r[o] = steps[t].r[j]; oa[o] = steps[t].oa[j]; ob[o] = steps[t].ob[j];
    }
  caps[0] = P.site_cap; caps[1] = P.env_cap; caps[2] = P.big_cap; caps[3] = P.mat_cap;
  caps[4] = P.env2_cap; caps[5] = P.slot_elems; caps[6] = P.slot_doubles;
  // region offsets in layout order, for the overlap check
  const int64_t offs[] = {P.off_dn, P.off_up, P.off_rst, P.off_b0, P.off_b1, P.off_b2, P.off_y,
                          P.off_xj, P.off_vt, P.off_c0, P.off_c1, P.off_l1, P.off_r1, P.off_l2,
                          P.off_r2, P.off_alpha, P.off_inv, P.off_tmp, P.off_dnf, P.off_upf};
  for (int i = 0; i < 20; ++i) caps[7 + i] = offs[i];
  return 0;
}

}  // extern "C"
