// peps_plan.h -- bond dimensions of every boundary-MPS step and the
// per-slot workspace layout.  Plain data, filled on the host, read by the
// kernels.
//
// Truncation (Fig. 1(c) of PEPS++): when a row is absorbed into an
// environment with site bonds (a_j, b_j), site j gets left bond
// A_j = a_j*Dl_j and right bond B_j = b_j*Dr_j (Dl_0 = Dr_{L-1} = 1, else D).
// A left-to-right QR sweep gives ranks r_{-1} = 1,
// r_j = min(r_{j-1}*Q, B_j); the right-to-left SVD sweep keeps
// c_L = 1, c_j = min(Dc, r_{j-1}, Q*c_{j+1}) singular values, so the
// truncated site j has dims (c_j, Q, c_{j+1}) (site 0: (1, Q, c_1)).
// These depend only on (L, D, Dc) and the number of rows already absorbed,
// and are the same for the upper and the lower environments.
#pragma once
#include <stdint.h>

// Resident blocks per SM the kernels' register budget is set for (their
// __launch_bounds__); the default slot count is this many per SM.
#ifndef PEPS_MINB
#define PEPS_MINB 2
#endif

#define PEPS_MAXL 32

struct PepsStep {
  // input environment site dims (left bond, physical, right bond)
  int16_t ia[PEPS_MAXL], ip[PEPS_MAXL], ib[PEPS_MAXL];
  // QR ranks r_j, j = 0..L-2 (r_{-1} = 1 implicit)
  int16_t r[PEPS_MAXL];
  // output site dims
  int16_t oa[PEPS_MAXL], ob[PEPS_MAXL];
};

struct PepsPlan {
  int32_t L, D, Dc, N;
  int32_t D2, D3, D4;
  int32_t nbonds;
  double J1, J2;
  int32_t nsteps;  // L - 1 absorption steps (U_0..U_{L-2} / Dn_{L-1}..Dn_1)
  // element counts / capacities (in scalars of the form's type)
  int64_t site_cap;   // Dc*D*Dc: capacity of one MPS site
  int64_t env_cap;    // L*site_cap
  int64_t big_cap;    // Dc^2 D^3: largest temporary
  int64_t mat_cap;    // (Dc*D)^2
  int64_t env2_cap;   // Dc*D*D*Dc: two-row strip environment
  // per-slot workspace offsets in scalars of the form's type
  int64_t off_dn, off_up, off_rst, off_b0, off_b1, off_b2, off_y, off_xj,
      off_vt, off_c0, off_c1, off_l1, off_r1, off_l2, off_r2, off_alpha, off_inv, off_tmp;
  int64_t slot_elems;  // scalars per slot
  // per-slot workspace offsets in doubles
  int64_t doff_scale, doff_delta, doff_alpha;
  int64_t slot_doubles;
};
