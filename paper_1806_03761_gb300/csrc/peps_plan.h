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
#include <string.h>

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
      off_vt, off_c0, off_c1, off_l1, off_r1, off_l2, off_r2, off_alpha, off_inv, off_tmp,
      off_dnf, off_upf;
  int64_t slot_elems;  // scalars per slot
  // per-slot workspace offsets in doubles
  int64_t doff_scale, doff_delta, doff_alpha;
  int64_t slot_doubles;
};

// ---------------------------------------------------------------------------
// Host-side construction of the plan (one place for every entry point).
// ---------------------------------------------------------------------------
static inline int64_t peps_up32(int64_t x) { return (x + 31) & ~int64_t(31); }
static inline int peps_imin(int a, int b) { return a < b ? a : b; }

// The bond dimensions of every absorption step t = 0 .. L-2 (the recurrences
// at the top of this file) into steps[0 .. L-2], and the scalar fields of P.
static inline void peps_plan_steps(int L, int D, int Dc, double J1, double J2, PepsPlan* P,
                                   PepsStep* steps) {
  memset(P, 0, sizeof(*P));
  P->L = L; P->D = D; P->Dc = Dc; P->N = L * L;
  P->D2 = D * D; P->D3 = D * D * D; P->D4 = D * D * D * D;
  P->nbonds = 2 * L * (L - 1) + 2 * (L - 1) * (L - 1);
  P->J1 = J1; P->J2 = J2;
  P->nsteps = L - 1;
  const int Q = D;
  for (int t = 0; t < L - 1; ++t) {
    PepsStep& st = steps[t];
    memset(&st, 0, sizeof(st));
    for (int j = 0; j < L; ++j) {
      if (t == 0) { st.ia[j] = 1; st.ip[j] = 1; st.ib[j] = 1; }
      else { st.ia[j] = steps[t - 1].oa[j]; st.ip[j] = (int16_t)D; st.ib[j] = steps[t - 1].ob[j]; }
    }
    int rprev = 1;
    for (int j = 0; j < L - 1; ++j) {
      const int r = peps_imin(rprev * Q, st.ib[j] * D);  // B_j = b_j * Dr_j, Dr_j = D for j < L-1
      st.r[j] = (int16_t)r;
      rprev = r;
    }
    int cn = 1;
    for (int j = L - 1; j >= 1; --j) {
      const int k = peps_imin(Dc, peps_imin((int)st.r[j - 1], Q * cn));
      st.oa[j] = (int16_t)k;
      st.ob[j] = (int16_t)cn;
      cn = k;
    }
    st.oa[0] = 1;
    st.ob[0] = (int16_t)cn;
  }
}

// The per-slot workspace layout.  amplitude_only: the amplitude-only kernel
// (lower environments and the row-0 one-row strip) needs neither the two-row
// strip environments nor the Delta staging; they are left out (offset 0).
static inline void peps_plan_layout(PepsPlan* P, bool amplitude_only) {
  const int L = P->L, D = P->D, Dc = P->Dc;
  P->site_cap = (int64_t)Dc * D * Dc;
  P->env_cap = (int64_t)L * P->site_cap;
  P->big_cap = (int64_t)Dc * Dc * D * D * D;
  P->mat_cap = (int64_t)(Dc * D) * (Dc * D);
  P->env2_cap = (int64_t)Dc * D * D * Dc;
  int64_t o = 0;
  auto take = [&](int64_t n) { int64_t r = o; o += peps_up32(n); return r; };
  P->off_dn = take((int64_t)(L + 1) * P->env_cap);
  P->off_up = take(3 * P->env_cap);
  P->off_rst = take((int64_t)L * P->mat_cap);
  P->off_b0 = take(P->big_cap);
  P->off_b1 = take(P->big_cap);
  P->off_b2 = take(P->big_cap);
  P->off_y = take(P->mat_cap);
  P->off_xj = take(P->mat_cap);
  P->off_vt = take(P->site_cap > P->D4 ? P->site_cap : (int64_t)P->D4);
  P->off_c0 = take(P->site_cap);
  P->off_c1 = take(P->site_cap);
  P->off_l1 = take((int64_t)(L + 1) * P->site_cap);
  P->off_r1 = take((int64_t)(L + 1) * P->site_cap);
  P->off_l2 = amplitude_only ? 0 : take((int64_t)(L + 1) * P->env2_cap);
  P->off_r2 = amplitude_only ? 0 : take((int64_t)(L + 1) * P->env2_cap);
  P->off_alpha = take(3 * (int64_t)Dc * D + 16);
  P->off_inv = take(13 * (int64_t)Dc * Dc * D);
  P->off_tmp = take(32);
  // environments of a configuration with one spin flipped (correlations)
  P->off_dnf = amplitude_only ? 0 : take((int64_t)(L + 1) * P->env_cap);
  P->off_upf = amplitude_only ? 0 : take(3 * P->env_cap);
  P->slot_elems = o;
  int64_t d = 0;
  auto taked = [&](int64_t n) { int64_t r = d; d += peps_up32(n); return r; };
  P->doff_scale = taked(4 * (L + 1));
  P->doff_delta = amplitude_only ? 0 : taked((int64_t)P->N * P->D4);
  P->doff_alpha = amplitude_only ? 0 : taked((int64_t)Dc * D + 8);
  P->slot_doubles = d;
}
