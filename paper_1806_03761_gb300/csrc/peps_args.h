// peps_args.h -- kernel argument blocks, shared by the launchers and the C ABI.
#pragma once
#include <stdint.h>
#include "peps_arith.cuh"
#include "peps_plan.h"

template <class R>
struct EvalArgs {
  PepsPlan P;
  const PepsStep* steps;
  const R* As;            // site tensors in the form's type
  const uint8_t* spins;   // [B][N]
  int64_t B;
  int want_energy, want_delta;
  const double* e_in;     // [B] energies for the Delta*E sums (logderiv only)
  double* e_loc;          // [B] or null
  double* log_abs;        // [B] or null
  int8_t* sign;           // [B] or null
  double* ratios;         // [B][nbonds] or null
  int32_t* n_flips;       // [B] or null
  double* delta;          // [B][N][D4] or null
  R* ws;                  // slot workspaces, P.slot_elems each
  double* wsd;            // slot double workspaces, P.slot_doubles each
  double* psum;           // slot partial sums: [slot][2*N*2*D4 + 1]
  int* flags;
};

template <class R>
struct SampleArgs {
  PepsPlan P;
  const PepsStep* steps;
  const R* As;
  uint32_t k0, k1;           // Philox key = seed
  int64_t n_chains, chain_offset;
  int n_burn, n_thin, spc;
  uint64_t first_sweep;
  const uint32_t* sweep_dev;  // nullable: the fused step's sweep number, read at run time
  uint8_t* out;              // [n_chains*spc][N]
  uint8_t* state;            // [n_chains][N] or null (in/out)
  int64_t* accepted;         // [n_chains] or null
  R* ws;
  double* wsd;
  int* flags;
};

// Spin correlations: items (sample b, source q), b < B, q < n_src.
template <class R>
struct CorrArgs {
  PepsPlan P;
  const PepsStep* steps;
  const R* As;
  const uint8_t* spins;   // [B][N]
  int64_t B;
  int n_src;
  const int32_t* src;     // [n_src] source sites, validated on the host
  double* ss;             // [B][n_src][N] local values of S_src . S_m
  R* ws;
  double* wsd;
  int* flags;
};

// One job of a multi-job launch (peps_multi_kernel): the job's evaluation
// arguments and the number of its first (job, sample) item.
template <class R>
struct MultiJobDev {
  EvalArgs<R> a;
  int64_t first_item;
};
