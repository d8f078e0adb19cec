// peps_api.cu -- the C ABI of libpeps.so (declared in include/peps.h):
// context and workspace management, argument checks, kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/peps.h"
#include "peps_args.h"
#include "peps_launch.h"

struct peps_ctx {
  peps_shape shape;
  PepsPlan plan;
  std::vector<PepsStep> steps_h;
  PepsStep* steps = nullptr;
  void* As = nullptr;      // site tensors in the form's type
  void* ws = nullptr;      // slot workspaces
  double* wsd = nullptr;   // slot double workspaces
  double* psum = nullptr;  // slot partial sums
  int* flags = nullptr;
  int32_t* idx = nullptr;  // 3N int32: correlation sources, bulk positions, bulk sites
  // device staging of the host-buffer VMC step (grown on demand)
  uint8_t* h_state = nullptr;
  double* h_out = nullptr;  // e_loc [n], log_abs [n]
  int8_t* h_sign = nullptr;
  double* h_sums = nullptr; // sum_delta, sum_delta_e, sum_e
  int64_t h_cap = 0;
  int nslots = 0;
  int tensors_set = 0;
  int device = 0;
  std::string err;
};

namespace {

int fail(peps_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(peps_ctx* c, cudaError_t e, const char* what) {
  return fail(c, PEPS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool shape_ok(const peps_shape* s, std::string* why) {
  if (!s) { *why = "shape is NULL"; return false; }
  if (s->L < 2 || s->L > PEPS_MAXL) { *why = "L must be in [2, 32]"; return false; }
  if (s->D < 1 || s->D > 8) { *why = "D must be in [1, 8]"; return false; }
  if (s->Dc < 1 || s->Dc * s->D > 256) { *why = "Dc must be >= 1 with Dc*D <= 256"; return false; }
  if (s->precision != PEPS_FP64 && s->precision != PEPS_MIXED && s->precision != PEPS_FP32) {
    *why = "precision must be PEPS_FP64, PEPS_MIXED or PEPS_FP32";
    return false;
  }
  if (!std::isfinite(s->J1) || !std::isfinite(s->J2)) { *why = "J1, J2 must be finite"; return false; }
  return true;
}

cudaError_t launch_eval_form(const EvalArgs<double>& a, int g, cudaStream_t s) { return peps_launch_eval_f64(a, g, s); }
cudaError_t launch_eval_form(const EvalArgs<ff>& a, int g, cudaStream_t s) { return peps_launch_eval_ff(a, g, s); }
cudaError_t launch_eval_form(const EvalArgs<float>& a, int g, cudaStream_t s) { return peps_launch_eval_f32(a, g, s); }
cudaError_t launch_sample_form(const SampleArgs<double>& a, int g, cudaStream_t s) { return peps_launch_sample_f64(a, g, s); }
cudaError_t launch_sample_form(const SampleArgs<ff>& a, int g, cudaStream_t s) { return peps_launch_sample_ff(a, g, s); }
cudaError_t launch_sample_form(const SampleArgs<float>& a, int g, cudaStream_t s) { return peps_launch_sample_f32(a, g, s); }
cudaError_t launch_vmc_form(const EvalArgs<double>& a, const SampleArgs<double>& b, int g, cudaStream_t s) { return peps_launch_vmc_f64(a, b, g, s); }
cudaError_t launch_vmc_form(const EvalArgs<ff>& a, const SampleArgs<ff>& b, int g, cudaStream_t s) { return peps_launch_vmc_ff(a, b, g, s); }
cudaError_t launch_vmc_form(const EvalArgs<float>& a, const SampleArgs<float>& b, int g, cudaStream_t s) { return peps_launch_vmc_f32(a, b, g, s); }
cudaError_t launch_corr_form(const CorrArgs<double>& a, int g, cudaStream_t s) { return peps_launch_corr_f64(a, g, s); }
cudaError_t launch_corr_form(const CorrArgs<ff>& a, int g, cudaStream_t s) { return peps_launch_corr_ff(a, g, s); }

// Bond dimensions of every absorption step and the slot layout (peps_plan.h).
void make_plan(const peps_shape& s, int nslots, PepsPlan* P, std::vector<PepsStep>* steps) {
  steps->assign(s.L - 1, PepsStep());
  peps_plan_steps(s.L, s.D, s.Dc, s.J1, s.J2, P, steps->data());
  peps_plan_layout(P, false);
  (void)nslots;
}

int64_t psum_len(const PepsPlan& P) { return 2 * (int64_t)P.N * 2 * P.D4 + 1; }

size_t elem_size(int precision) {
  return precision == PEPS_FP64 ? sizeof(double) : precision == PEPS_FP32 ? sizeof(float) : sizeof(ff);
}

int default_slots() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return PEPS_MINB * sms;
}

template <class R>
int launch_eval(peps_ctx* c, const uint8_t* spins, int64_t B, int energy, int delta_on,
                const double* e_in, double* e_loc, double* log_abs, int8_t* sign,
                double* ratios, int32_t* n_flips, double* delta, double* sd, double* sde,
                double* se, int accumulate, cudaStream_t st) {
  EvalArgs<R> a;
  a.P = c->plan;
  a.steps = c->steps;
  a.As = static_cast<const R*>(c->As);
  a.spins = spins;
  a.B = B;
  a.want_energy = energy;
  a.want_delta = delta_on;
  a.e_in = e_in;
  a.e_loc = e_loc;
  a.log_abs = log_abs;
  a.sign = sign;
  a.ratios = ratios;
  a.n_flips = n_flips;
  a.delta = delta;
  a.ws = static_cast<R*>(c->ws);
  a.wsd = c->wsd;
  a.psum = c->psum;
  a.flags = c->flags;
  int grid = (int)std::min<int64_t>(c->nslots, B);
  cudaError_t e = launch_eval_form(a, grid, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_eval_kernel launch");
  if (delta_on) {
    int64_t len = psum_len(c->plan);
    e = peps_launch_reduce(c->psum, grid, len, sd, sde, se, accumulate, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "peps_reduce_slots launch");
  }
  return PEPS_OK;
}

int eval_common(peps_ctx* c, const uint8_t* spins, int64_t B, int energy, int delta_on,
                const double* e_in, double* e_loc, double* log_abs, int8_t* sign,
                double* ratios, int32_t* n_flips, double* delta, double* sd, double* sde,
                double* se, int accumulate, void* stream) {
  if (!c) return PEPS_EINVAL;
  if (B < 0) return fail(c, PEPS_EINVAL, "B must be >= 0");
  if (!c->tensors_set) return fail(c, PEPS_EINVAL, "peps_set_tensors has not been called");
  if (B > 0 && !spins) return fail(c, PEPS_EINVAL, "spins is NULL");
  if (delta_on && (!sd || !sde || !se)) return fail(c, PEPS_EINVAL, "sum_delta, sum_delta_e and sum_e are required");
  if (delta_on && !energy && B > 0 && !e_in) return fail(c, PEPS_EINVAL, "e_loc is NULL");
  if (accumulate != 0 && accumulate != 1) return fail(c, PEPS_EINVAL, "accumulate must be 0 or 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  if (B == 0) {
    if (delta_on && !accumulate) {
      size_t n = (size_t)c->plan.N * 2 * c->plan.D4 * sizeof(double);
      cudaError_t e1 = cudaMemsetAsync(sd, 0, n, st);
      cudaError_t e2 = cudaMemsetAsync(sde, 0, n, st);
      cudaError_t e3 = cudaMemsetAsync(se, 0, sizeof(double), st);
      if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
        return fail(c, PEPS_ECUDA, "cudaMemsetAsync failed");
    }
    return PEPS_OK;
  }
  if (c->shape.precision == PEPS_FP64)
    return launch_eval<double>(c, spins, B, energy, delta_on, e_in, e_loc, log_abs, sign, ratios,
                               n_flips, delta, sd, sde, se, accumulate, st);
  if (c->shape.precision == PEPS_FP32)
    return launch_eval<float>(c, spins, B, energy, delta_on, e_in, e_loc, log_abs, sign, ratios,
                              n_flips, delta, sd, sde, se, accumulate, st);
  return launch_eval<ff>(c, spins, B, energy, delta_on, e_in, e_loc, log_abs, sign, ratios,
                         n_flips, delta, sd, sde, se, accumulate, st);
}


template <class R>
int launch_sample(peps_ctx* c, uint64_t seed, int64_t n_chains, int64_t chain_offset,
                  int32_t n_burn, int32_t n_thin, int32_t spc, uint64_t first_sweep,
                  uint8_t* out, uint8_t* state, int64_t* accepted, cudaStream_t st) {
  SampleArgs<R> a;
  a.P = c->plan;
  a.steps = c->steps;
  a.As = static_cast<const R*>(c->As);
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.n_chains = n_chains;
  a.chain_offset = chain_offset;
  a.n_burn = n_burn;
  a.n_thin = n_thin;
  a.spc = spc;
  a.first_sweep = first_sweep;
  a.out = out;
  a.state = state;
  a.accepted = accepted;
  a.ws = static_cast<R*>(c->ws);
  a.wsd = c->wsd;
  a.flags = c->flags;
  int grid = (int)std::min<int64_t>(c->nslots, n_chains);
  cudaError_t e = launch_sample_form(a, grid, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_sample_kernel launch");
  return PEPS_OK;
}

template <class R>
int launch_vmc(peps_ctx* c, uint64_t seed, int64_t n, int64_t chain_offset, uint64_t sweep,
               const uint32_t* sweep_dev, uint8_t* state, double* e_loc, double* log_abs,
               int8_t* sign, double* sd, double* sde, double* se, int accumulate,
               int64_t* accepted, cudaStream_t st) {
  EvalArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.P = c->plan;
  a.steps = c->steps;
  a.As = static_cast<const R*>(c->As);
  a.B = n;
  a.want_energy = 1;
  a.want_delta = 1;
  a.e_loc = e_loc;
  a.log_abs = log_abs;
  a.sign = sign;
  a.ws = static_cast<R*>(c->ws);
  a.wsd = c->wsd;
  a.psum = c->psum;
  a.flags = c->flags;
  SampleArgs<R> s;
  std::memset(&s, 0, sizeof(s));
  s.k0 = (uint32_t)seed;
  s.k1 = (uint32_t)(seed >> 32);
  s.n_chains = n;
  s.chain_offset = chain_offset;
  s.first_sweep = sweep;
  s.sweep_dev = sweep_dev;
  s.state = state;
  s.accepted = accepted;
  int grid = (int)std::min<int64_t>(c->nslots, n);
  cudaError_t e = launch_vmc_form(a, s, grid, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_vmc_kernel launch");
  e = peps_launch_reduce(c->psum, grid, psum_len(c->plan), sd, sde, se, accumulate, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_reduce_slots launch");
  return PEPS_OK;
}

template <class R>
int launch_corr(peps_ctx* c, const uint8_t* spins, int64_t B, int32_t n_src, double* ss,
                cudaStream_t st) {
  CorrArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.P = c->plan;
  a.steps = c->steps;
  a.As = static_cast<const R*>(c->As);
  a.spins = spins;
  a.B = B;
  a.n_src = n_src;
  a.src = c->idx;
  a.ss = ss;
  a.ws = static_cast<R*>(c->ws);
  a.wsd = c->wsd;
  a.flags = c->flags;
  int grid = (int)std::min<int64_t>(c->nslots, B * n_src);
  cudaError_t e = launch_corr_form(a, grid, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_corr_kernel launch");
  return PEPS_OK;
}

// The central (L-4) x (L-4) sites, every site when L <= 4.
std::vector<int32_t> bulk_list(int L) {
  const int lo = L > 4 ? 2 : 0, hi = L > 4 ? L - 2 : L;
  std::vector<int32_t> b;
  for (int i = lo; i < hi; ++i)
    for (int j = lo; j < hi; ++j) b.push_back(i * L + j);
  return b;
}

}  // namespace

extern "C" {

size_t peps_workspace_bytes(const peps_shape* shape, int32_t slots) {
  std::string why;
  if (!shape_ok(shape, &why) || slots < 0) return 0;
  if (slots == 0) slots = default_slots();
  PepsPlan P;
  std::vector<PepsStep> st;
  make_plan(*shape, slots, &P, &st);
  size_t es = elem_size(shape->precision);
  return (size_t)slots * ((size_t)P.slot_elems * es + (size_t)P.slot_doubles * 8 +
                          (size_t)psum_len(P) * 8) +
         (size_t)P.N * 2 * P.D4 * es + st.size() * sizeof(PepsStep);
}

int peps_slots(const peps_ctx* c, int32_t* slots) {
  if (!c || !slots) return PEPS_EINVAL;
  *slots = c->nslots;
  return PEPS_OK;
}

int peps_phase_cycles(const peps_ctx* c, uint64_t* out, int32_t n, int32_t* n_phases) {
  if (!c || !n_phases || n < 0 || (n > 0 && !out)) return PEPS_EINVAL;
  unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
  *n_phases = c->shape.precision == PEPS_FP64 ? peps_phase_read_f64(o, n)
              : c->shape.precision == PEPS_FP32 ? peps_phase_read_f32(o, n)
                                                : peps_phase_read_ff(o, n);
  return PEPS_OK;
}

int peps_create(const peps_shape* shape, int32_t slots, peps_ctx** out) {
  if (!out) return PEPS_EINVAL;
  *out = nullptr;
  std::string why;
  if (!shape_ok(shape, &why)) return PEPS_EINVAL;
  if (slots < 0) return PEPS_EINVAL;
  peps_ctx* c = new (std::nothrow) peps_ctx();
  if (!c) return PEPS_ENOMEM;
  c->shape = *shape;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return PEPS_ECUDA; }
  if (slots == 0) slots = default_slots();
  if (slots <= 0) { delete c; return PEPS_ECUDA; }
  c->nslots = slots;
  make_plan(*shape, slots, &c->plan, &c->steps_h);
  const PepsPlan& P = c->plan;
  size_t es = elem_size(shape->precision);
  bool ok = cudaMalloc(&c->steps, c->steps_h.size() * sizeof(PepsStep)) == cudaSuccess &&
            cudaMalloc(&c->As, (size_t)P.N * 2 * P.D4 * es) == cudaSuccess &&
            cudaMalloc(&c->ws, (size_t)slots * P.slot_elems * es) == cudaSuccess &&
            cudaMalloc(&c->wsd, (size_t)slots * P.slot_doubles * 8) == cudaSuccess &&
            cudaMalloc(&c->psum, (size_t)slots * psum_len(P) * 8) == cudaSuccess &&
            cudaMalloc(&c->flags, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->idx, 3 * (size_t)P.N * sizeof(int32_t)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    peps_destroy(c);
    return PEPS_ENOMEM;
  }
  if (cudaMemcpy(c->steps, c->steps_h.data(), c->steps_h.size() * sizeof(PepsStep),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->flags, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->ws, 0, (size_t)slots * P.slot_elems * es) != cudaSuccess) {
    peps_destroy(c);
    return PEPS_ECUDA;
  }
  *out = c;
  return PEPS_OK;
}

int peps_destroy(peps_ctx* c) {
  if (!c) return PEPS_EINVAL;
  cudaFree(c->steps);
  cudaFree(c->As);
  cudaFree(c->ws);
  cudaFree(c->wsd);
  cudaFree(c->psum);
  cudaFree(c->flags);
  cudaFree(c->idx);
  cudaFree(c->h_state);
  cudaFree(c->h_out);
  cudaFree(c->h_sign);
  cudaFree(c->h_sums);
  delete c;
  return PEPS_OK;
}

const char* peps_last_error(const peps_ctx* c) { return c ? c->err.c_str() : "no context"; }

int peps_set_tensors(peps_ctx* c, const double* A, void* stream) {
  if (!c) return PEPS_EINVAL;
  if (!A) return fail(c, PEPS_EINVAL, "A is NULL");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  int64_t n = (int64_t)c->plan.N * 2 * c->plan.D4;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = peps_launch_convert(c->shape.precision, A, c->As, n, c->flags, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_convert_kernel launch");
  c->tensors_set = 1;
  return PEPS_OK;
}

int peps_amplitudes(peps_ctx* c, const uint8_t* spins, int64_t B, double* log_abs,
                    int8_t* sign, void* stream) {
  if (c && B > 0 && (!log_abs || !sign)) return fail(c, PEPS_EINVAL, "log_abs and sign are required");
  return eval_common(c, spins, B, 0, 0, nullptr, nullptr, log_abs, sign, nullptr, nullptr,
                     nullptr, nullptr, nullptr, nullptr, 0, stream);
}

int peps_local_energy(peps_ctx* c, const uint8_t* spins, int64_t B, double* e_loc,
                      double* log_abs, int8_t* sign, double* ratios, int32_t* n_flips,
                      void* stream) {
  if (c && B > 0 && !e_loc) return fail(c, PEPS_EINVAL, "e_loc is NULL");
  return eval_common(c, spins, B, 1, 0, nullptr, e_loc, log_abs, sign, ratios, n_flips,
                     nullptr, nullptr, nullptr, nullptr, 0, stream);
}

int peps_logderiv(peps_ctx* c, const uint8_t* spins, int64_t B, const double* e_loc,
                  double* delta, double* sum_delta, double* sum_delta_e, double* sum_e,
                  int32_t accumulate, void* stream) {
  return eval_common(c, spins, B, 0, 1, e_loc, nullptr, nullptr, nullptr, nullptr, nullptr,
                     delta, sum_delta, sum_delta_e, sum_e, accumulate, stream);
}

int peps_evaluate(peps_ctx* c, const uint8_t* spins, int64_t B, double* e_loc, double* log_abs,
                  int8_t* sign, double* ratios, int32_t* n_flips, double* delta,
                  double* sum_delta, double* sum_delta_e, double* sum_e, int32_t accumulate,
                  void* stream) {
  if (c && B > 0 && !e_loc) return fail(c, PEPS_EINVAL, "e_loc is NULL");
  return eval_common(c, spins, B, 1, 1, nullptr, e_loc, log_abs, sign, ratios, n_flips, delta,
                     sum_delta, sum_delta_e, sum_e, accumulate, stream);
}

int peps_grad_step(peps_ctx* c, const double* sum_delta, const double* sum_delta_e,
                   const double* sum_e, int64_t M, double dt, uint64_t seed, uint64_t step,
                   double* A_inout, void* stream) {
  if (!c) return PEPS_EINVAL;
  if (!sum_delta || !sum_delta_e || !sum_e || !A_inout) return fail(c, PEPS_EINVAL, "NULL argument");
  if (M <= 0) return fail(c, PEPS_EINVAL, "M must be positive");
  if (step >> 32) return fail(c, PEPS_EINVAL, "step must be < 2^32");
  if (!std::isfinite(dt)) return fail(c, PEPS_EINVAL, "dt must be finite");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  int64_t n = (int64_t)c->plan.N * 2 * c->plan.D4;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  cudaError_t e = peps_launch_grad(c->shape.precision, sum_delta, sum_delta_e, sum_e, (double)M, dt,
                                   k0, k1, (uint32_t)step, nullptr, A_inout, c->As, n, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_grad_kernel launch");
  c->tensors_set = 1;
  return PEPS_OK;
}

int peps_sample_batch(peps_ctx* c, uint64_t seed, int64_t n_chains, int64_t chain_offset,
                      int32_t n_burn, int32_t n_thin, int32_t samples_per_chain,
                      uint64_t first_sweep, uint8_t* spins_out, uint8_t* chain_state,
                      int64_t* accepted, void* stream) {
  if (!c) return PEPS_EINVAL;
  if (n_chains < 0 || n_burn < 0 || n_thin < 1 || samples_per_chain < 0)
    return fail(c, PEPS_EINVAL, "need n_chains >= 0, n_burn >= 0, n_thin >= 1, samples_per_chain >= 0");
  if (chain_offset < 0 || chain_offset + n_chains > (int64_t(1) << 32))
    return fail(c, PEPS_EINVAL, "chain indices must lie in [0, 2^32)");
  int64_t total = (int64_t)n_burn + (int64_t)samples_per_chain * n_thin;
  if (first_sweep + (uint64_t)total > (uint64_t(1) << 32))
    return fail(c, PEPS_EINVAL, "sweep numbers must lie in [0, 2^32)");
  if (n_chains > 0 && samples_per_chain > 0 && !spins_out) return fail(c, PEPS_EINVAL, "spins_out is NULL");
  if (!c->tensors_set) return fail(c, PEPS_EINVAL, "peps_set_tensors has not been called");
  if (n_chains == 0) return PEPS_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->shape.precision == PEPS_FP64)
    return launch_sample<double>(c, seed, n_chains, chain_offset, n_burn, n_thin, samples_per_chain,
                                 first_sweep, spins_out, chain_state, accepted, st);
  if (c->shape.precision == PEPS_FP32)
    return launch_sample<float>(c, seed, n_chains, chain_offset, n_burn, n_thin, samples_per_chain,
                                first_sweep, spins_out, chain_state, accepted, st);
  return launch_sample<ff>(c, seed, n_chains, chain_offset, n_burn, n_thin, samples_per_chain,
                           first_sweep, spins_out, chain_state, accepted, st);
}

}  // extern "C"

namespace {
int vmc_common(peps_ctx* c, uint64_t seed, int64_t n_chains, int64_t chain_offset,
               uint64_t sweep, const uint32_t* sweep_dev, uint8_t* chain_state, double* e_loc,
               double* log_abs, int8_t* sign, double* sum_delta, double* sum_delta_e,
               double* sum_e, int32_t accumulate, int64_t* accepted, void* stream) {
  if (!c) return PEPS_EINVAL;
  if (n_chains < 0) return fail(c, PEPS_EINVAL, "n_chains must be >= 0");
  if (chain_offset < 0 || chain_offset + n_chains > (int64_t(1) << 32))
    return fail(c, PEPS_EINVAL, "chain indices must lie in [0, 2^32)");
  if (sweep >= (uint64_t(1) << 32)) return fail(c, PEPS_EINVAL, "sweep must be < 2^32");
  if (accumulate != 0 && accumulate != 1) return fail(c, PEPS_EINVAL, "accumulate must be 0 or 1");
  if (!sum_delta || !sum_delta_e || !sum_e) return fail(c, PEPS_EINVAL, "sum_delta, sum_delta_e and sum_e are required");
  if (!c->tensors_set) return fail(c, PEPS_EINVAL, "peps_set_tensors has not been called");
  if (n_chains == 0) return eval_common(c, nullptr, 0, 1, 1, nullptr, nullptr, nullptr, nullptr, nullptr,
                                        nullptr, nullptr, sum_delta, sum_delta_e, sum_e, accumulate, stream);
  if (!chain_state || !e_loc) return fail(c, PEPS_EINVAL, "chain_state and e_loc are required");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->shape.precision == PEPS_FP64)
    return launch_vmc<double>(c, seed, n_chains, chain_offset, sweep, sweep_dev, chain_state, e_loc,
                              log_abs, sign, sum_delta, sum_delta_e, sum_e, accumulate, accepted, st);
  if (c->shape.precision == PEPS_FP32)
    return launch_vmc<float>(c, seed, n_chains, chain_offset, sweep, sweep_dev, chain_state, e_loc,
                             log_abs, sign, sum_delta, sum_delta_e, sum_e, accumulate, accepted, st);
  return launch_vmc<ff>(c, seed, n_chains, chain_offset, sweep, sweep_dev, chain_state, e_loc,
                        log_abs, sign, sum_delta, sum_delta_e, sum_e, accumulate, accepted, st);
}
}  // namespace

extern "C" {

int peps_vmc_step(peps_ctx* c, uint64_t seed, int64_t n_chains, int64_t chain_offset,
                  uint64_t sweep, uint8_t* chain_state, double* e_loc, double* log_abs,
                  int8_t* sign, double* sum_delta, double* sum_delta_e, double* sum_e,
                  int32_t accumulate, int64_t* accepted, void* stream) {
  return vmc_common(c, seed, n_chains, chain_offset, sweep, nullptr, chain_state, e_loc, log_abs,
                    sign, sum_delta, sum_delta_e, sum_e, accumulate, accepted, stream);
}

int peps_vmc_step_host(peps_ctx* c, uint64_t seed, int64_t n_chains, int64_t chain_offset,
                       uint64_t sweep, uint8_t* chain_state, double* e_loc, double* log_abs,
                       int8_t* sign, double* sum_e, double* sum_delta, double* sum_delta_e,
                       double* sum_e_dev, void* stream) {
  if (!c) return PEPS_EINVAL;
  if (n_chains < 1) return fail(c, PEPS_EINVAL, "n_chains must be >= 1");
  if (!chain_state || !e_loc) return fail(c, PEPS_EINVAL, "chain_state and e_loc are required");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  const int64_t N = c->plan.N;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_chains > c->h_cap) {  // staging grown (allocation: before any timed use)
    cudaFree(c->h_state);
    cudaFree(c->h_out);
    cudaFree(c->h_sign);
    c->h_state = nullptr; c->h_out = nullptr; c->h_sign = nullptr;
    c->h_cap = 0;
    if (cudaMalloc(&c->h_state, (size_t)n_chains * N) != cudaSuccess ||
        cudaMalloc(&c->h_out, (size_t)n_chains * 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->h_sign, (size_t)n_chains) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, PEPS_ENOMEM, "staging of the host-buffer step");
    }
    c->h_cap = n_chains;
  }
  double* sd = sum_delta;
  double* sde = sum_delta_e;
  double* se = sum_e_dev;
  if (!sd || !sde || !se) {  // the context's own sums
    if (!c->h_sums &&
        cudaMalloc(&c->h_sums, (2 * (size_t)N * 2 * c->plan.D4 + 1) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, PEPS_ENOMEM, "gradient sums of the host-buffer step");
    }
    sd = c->h_sums;
    sde = sd + (size_t)N * 2 * c->plan.D4;
    se = sde + (size_t)N * 2 * c->plan.D4;
  }
  if (cudaMemcpyAsync(c->h_state, chain_state, (size_t)n_chains * N, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return fail(c, PEPS_ECUDA, "copying the chain states in");
  int rc = vmc_common(c, seed, n_chains, chain_offset, sweep, nullptr, c->h_state, c->h_out,
                      c->h_out + n_chains, c->h_sign, sd, sde, se, 0, nullptr, stream);
  if (rc != PEPS_OK) return rc;
  bool ok = cudaMemcpyAsync(chain_state, c->h_state, (size_t)n_chains * N, cudaMemcpyDeviceToHost, st) ==
                cudaSuccess &&
            cudaMemcpyAsync(e_loc, c->h_out, (size_t)n_chains * sizeof(double), cudaMemcpyDeviceToHost,
                            st) == cudaSuccess;
  if (ok && log_abs)
    ok = cudaMemcpyAsync(log_abs, c->h_out + n_chains, (size_t)n_chains * sizeof(double),
                         cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (ok && sign)
    ok = cudaMemcpyAsync(sign, c->h_sign, (size_t)n_chains, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (ok && sum_e)
    ok = cudaMemcpyAsync(sum_e, se, sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (!ok) return fail(c, PEPS_ECUDA, "copying the results out");
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaStreamSynchronize");
  return PEPS_OK;
}

int peps_vmc_step_dc(peps_ctx* c, uint64_t seed, int64_t n_chains, int64_t chain_offset,
                     const uint32_t* counters, uint8_t* chain_state, double* e_loc,
                     double* log_abs, int8_t* sign, double* sum_delta, double* sum_delta_e,
                     double* sum_e, int32_t accumulate, int64_t* accepted, void* stream) {
  if (c && !counters) return fail(c, PEPS_EINVAL, "counters is NULL");
  return vmc_common(c, seed, n_chains, chain_offset, 0, counters, chain_state, e_loc, log_abs,
                    sign, sum_delta, sum_delta_e, sum_e, accumulate, accepted, stream);
}

int peps_grad_step_dc(peps_ctx* c, const double* sum_delta, const double* sum_delta_e,
                      const double* sum_e, int64_t M, double dt, uint64_t seed,
                      const uint32_t* counters, double* A_inout, void* stream) {
  if (!c) return PEPS_EINVAL;
  if (!sum_delta || !sum_delta_e || !sum_e || !A_inout || !counters)
    return fail(c, PEPS_EINVAL, "NULL argument");
  if (M <= 0) return fail(c, PEPS_EINVAL, "M must be positive");
  if (!std::isfinite(dt)) return fail(c, PEPS_EINVAL, "dt must be finite");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  int64_t n = (int64_t)c->plan.N * 2 * c->plan.D4;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = peps_launch_grad(c->shape.precision, sum_delta, sum_delta_e, sum_e, (double)M, dt,
                                   (uint32_t)seed, (uint32_t)(seed >> 32), 0, counters + 1, A_inout,
                                   c->As, n, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_grad_kernel launch");
  c->tensors_set = 1;
  return PEPS_OK;
}

int peps_counters_advance(uint32_t* counters, int32_t n, uint32_t inc, void* stream) {
  if (!counters || n < 1 || n > 64) return PEPS_EINVAL;
  return peps_launch_counters(counters, n, inc, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PEPS_OK : PEPS_ECUDA;
}

int peps_correlations(peps_ctx* c, const uint8_t* spins, int64_t B, int32_t n_src,
                      const int32_t* src, double* ss, double* ss_mean, void* stream) {
  if (!c) return PEPS_EINVAL;
  const int N = c->plan.N;
  if (B < 0) return fail(c, PEPS_EINVAL, "B must be >= 0");
  if (n_src < 1 || n_src > N || !src) return fail(c, PEPS_EINVAL, "need 1 <= n_src <= N sources");
  for (int q = 0; q < n_src; ++q)
    if (src[q] < 0 || src[q] >= N) return fail(c, PEPS_EINVAL, "source sites must lie in [0, N)");
  if (c->shape.precision == PEPS_FP32)
    return fail(c, PEPS_EINVAL, "correlations are computed in the FP64 and mixed forms");
  if (!c->tensors_set) return fail(c, PEPS_EINVAL, "peps_set_tensors has not been called");
  if (B == 0) return PEPS_OK;
  if (!spins || !ss) return fail(c, PEPS_EINVAL, "spins and ss are required");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(c->idx, src, (size_t)n_src * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the source sites");
  int rc = c->shape.precision == PEPS_FP64 ? launch_corr<double>(c, spins, B, n_src, ss, st)
                                           : launch_corr<ff>(c, spins, B, n_src, ss, st);
  if (rc != PEPS_OK || !ss_mean) return rc;
  e = peps_launch_corr_mean(ss, B, (int64_t)n_src * N, ss_mean, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_corr_mean launch");
  return PEPS_OK;
}

int peps_structure_factor(peps_ctx* c, const double* ss_mean, int32_t n_src, const int32_t* src,
                          double kx, double ky, double* m2, void* stream) {
  if (!c) return PEPS_EINVAL;
  const int L = c->plan.L, N = c->plan.N;
  if (!ss_mean || !m2 || !src || n_src < 1 || n_src > N)
    return fail(c, PEPS_EINVAL, "ss_mean, src (1 <= n_src <= N) and m2 are required");
  if (!std::isfinite(kx) || !std::isfinite(ky)) return fail(c, PEPS_EINVAL, "k must be finite");
  std::vector<int32_t> bulk = bulk_list(L), pos(bulk.size(), -1);
  for (size_t t = 0; t < bulk.size(); ++t)
    for (int q = 0; q < n_src; ++q)
      if (src[q] == bulk[t]) { pos[t] = q; break; }
  for (int32_t p : pos)
    if (p < 0) return fail(c, PEPS_EINVAL, "every bulk site must be among the sources");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = bulk.size() * sizeof(int32_t);
  cudaError_t e = cudaMemcpyAsync(c->idx + N, pos.data(), nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->idx + 2 * N, bulk.data(), nb, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the bulk sites");
  e = peps_launch_structure_factor(ss_mean, L, N, c->idx + N, (int)bulk.size(), c->idx + 2 * N,
                                   kx, ky, m2, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "peps_structure_factor launch");
  return PEPS_OK;
}

// ---------------------------------------------------------------------------
// Multi-job launches (jobs of different shapes, one precision form).
// ---------------------------------------------------------------------------
}  // extern "C"

struct peps_pool {
  int precision = 0;
  int nslots = 0;
  int max_jobs = 0;
  int device = 0;
  int64_t slot_elems = 0, slot_doubles = 0;
  void* ws = nullptr;
  double* wsd = nullptr;
  void* jobs = nullptr;               // MultiJobDev<R>[max_jobs]
  unsigned long long* next = nullptr; // the work-queue counter
  int* flags = nullptr;
};

namespace {

template <class R>
int launch_multi(peps_pool* pool, const peps_multi_job* jobs, int32_t n_jobs, cudaStream_t st) {
  // the costliest jobs first (per-sample cost ~ L^3 (D Dc)^3), so that their
  // long items start early and the cheap ones fill in behind them
  std::vector<int> order(n_jobs);
  for (int q = 0; q < n_jobs; ++q) order[q] = q;
  auto cost = [&](int q) {
    const PepsPlan& P = jobs[q].ctx->plan;
    const double x = (double)P.D * P.Dc;
    return (double)P.L * P.L * P.L * x * x * x;
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  std::vector<MultiJobDev<R>> h(n_jobs);
  int64_t items = 0;
  for (int k = 0; k < n_jobs; ++k) {
    const peps_multi_job& j = jobs[order[k]];
    MultiJobDev<R>& d = h[k];
    std::memset(&d, 0, sizeof(d));
    d.a.P = j.ctx->plan;
    d.a.steps = j.ctx->steps;
    d.a.As = static_cast<const R*>(j.ctx->As);
    d.a.spins = j.spins;
    d.a.B = j.B;
    d.a.want_energy = 1;
    d.a.e_loc = j.e_loc;
    d.a.log_abs = j.log_abs;
    d.a.sign = j.sign;
    d.a.ratios = j.ratios;
    d.a.n_flips = j.n_flips;
    d.a.flags = pool->flags;
    d.first_item = items;
    items += j.B;
  }
  if (items == 0) return PEPS_OK;
  // pageable source: the call returns once the bytes are staged
  if (cudaMemcpyAsync(pool->jobs, h.data(), h.size() * sizeof(MultiJobDev<R>), cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemsetAsync(pool->next, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return PEPS_ECUDA;
  const int grid = (int)std::min<int64_t>(pool->nslots, items);
  cudaError_t e;
  if (pool->precision == PEPS_FP64)
    e = peps_launch_multi_f64(static_cast<const MultiJobDev<double>*>(pool->jobs), n_jobs, items,
                              pool->next, static_cast<double*>(pool->ws), pool->wsd,
                              pool->slot_elems, pool->slot_doubles, pool->flags, grid, st);
  else
    e = peps_launch_multi_ff(static_cast<const MultiJobDev<ff>*>(pool->jobs), n_jobs, items,
                             pool->next, static_cast<ff*>(pool->ws), pool->wsd, pool->slot_elems,
                             pool->slot_doubles, pool->flags, grid, st);
  return e == cudaSuccess ? PEPS_OK : PEPS_ECUDA;
}

}  // namespace

extern "C" {

int peps_pool_create(int32_t precision, int32_t slots, const peps_shape* shapes, int32_t n_shapes,
                     int32_t max_jobs, peps_pool** out) {
  if (!out) return PEPS_EINVAL;
  *out = nullptr;
  if (precision != PEPS_FP64 && precision != PEPS_MIXED) return PEPS_EINVAL;
  if (!shapes || n_shapes < 1 || max_jobs < 1 || slots < 0) return PEPS_EINVAL;
  int64_t se = 0, sd = 0;
  for (int q = 0; q < n_shapes; ++q) {
    std::string why;
    if (!shape_ok(&shapes[q], &why) || shapes[q].precision != precision) return PEPS_EINVAL;
    PepsPlan P;
    std::vector<PepsStep> st;
    make_plan(shapes[q], 1, &P, &st);
    se = std::max(se, P.slot_elems);
    sd = std::max(sd, P.slot_doubles);
  }
  peps_pool* p = new (std::nothrow) peps_pool();
  if (!p) return PEPS_ENOMEM;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return PEPS_ECUDA; }
  p->precision = precision;
  p->nslots = slots > 0 ? slots : default_slots();
  p->max_jobs = max_jobs;
  p->slot_elems = se;
  p->slot_doubles = sd;
  const size_t es = elem_size(precision);
  const size_t jb = precision == PEPS_FP64 ? sizeof(MultiJobDev<double>) : sizeof(MultiJobDev<ff>);
  bool ok = p->nslots > 0 &&
            cudaMalloc(&p->ws, (size_t)p->nslots * se * es) == cudaSuccess &&
            cudaMalloc(&p->wsd, (size_t)p->nslots * sd * 8) == cudaSuccess &&
            cudaMalloc(&p->jobs, (size_t)max_jobs * jb) == cudaSuccess &&
            cudaMalloc(&p->next, sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&p->flags, sizeof(int)) == cudaSuccess;
  if (!ok || cudaMemset(p->flags, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(p->ws, 0, (size_t)p->nslots * se * es) != cudaSuccess) {
    cudaGetLastError();
    peps_pool_destroy(p);
    return PEPS_ENOMEM;
  }
  *out = p;
  return PEPS_OK;
}

int peps_pool_destroy(peps_pool* p) {
  if (!p) return PEPS_EINVAL;
  cudaFree(p->ws);
  cudaFree(p->wsd);
  cudaFree(p->jobs);
  cudaFree(p->next);
  cudaFree(p->flags);
  delete p;
  return PEPS_OK;
}

int peps_pool_slots(const peps_pool* p, int32_t* slots) {
  if (!p || !slots) return PEPS_EINVAL;
  *slots = p->nslots;
  return PEPS_OK;
}

int peps_local_energy_multi(peps_pool* pool, const peps_multi_job* jobs, int32_t n_jobs,
                            void* stream) {
  if (!pool || !jobs || n_jobs < 1 || n_jobs > pool->max_jobs) return PEPS_EINVAL;
  for (int q = 0; q < n_jobs; ++q) {
    const peps_multi_job& j = jobs[q];
    if (!j.ctx || !j.ctx->tensors_set || j.B < 0) return PEPS_EINVAL;
    if (j.ctx->shape.precision != pool->precision || j.ctx->device != pool->device) return PEPS_EINVAL;
    if (j.ctx->plan.slot_elems > pool->slot_elems || j.ctx->plan.slot_doubles > pool->slot_doubles)
      return PEPS_EINVAL;
    if (j.B > 0 && (!j.spins || !j.e_loc)) return PEPS_EINVAL;
  }
  if (cudaSetDevice(pool->device) != cudaSuccess) return PEPS_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return pool->precision == PEPS_FP64 ? launch_multi<double>(pool, jobs, n_jobs, st)
                                      : launch_multi<ff>(pool, jobs, n_jobs, st);
}

int peps_pool_sync_status(peps_pool* p, void* stream, int32_t* flags) {
  if (!p) return PEPS_EINVAL;
  if (cudaSetDevice(p->device) != cudaSuccess) return PEPS_ECUDA;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return PEPS_ECUDA;
  int h = 0;
  if (cudaMemcpy(&h, p->flags, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(p->flags, 0, sizeof(int)) != cudaSuccess)
    return PEPS_ECUDA;
  if (flags) *flags = h;
  return h ? PEPS_ENUMERIC : PEPS_OK;
}

int peps_sync_status(peps_ctx* c, void* stream, int32_t* flags) {
  if (!c) return PEPS_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PEPS_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  int h = 0;
  e = cudaMemcpy(&h, c->flags, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "reading the error flags");
  e = cudaMemset(c->flags, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(c, e, "clearing the error flags");
  if (flags) *flags = h;
  if (h) return fail(c, PEPS_ENUMERIC, "device-side numeric condition (see flags)");
  return PEPS_OK;
}

double peps_flops_per_sample(const peps_shape* shape, int32_t what) {
  std::string why;
  if (!shape_ok(shape, &why) || what < 0 || what > 2) return 0.0;
  PepsPlan P;
  std::vector<PepsStep> steps;
  make_plan(*shape, 1, &P, &steps);
  const int L = P.L, D = P.D;
  // one boundary-MPS compression (absorption + truncation) of step t
  auto compress_flops = [&](const PepsStep& st) {
    double f = 0.0;
    int rprev = 1;
    for (int j = 0; j < L - 1; ++j) {
      double a = st.ia[j], p = st.ip[j], b = st.ib[j];
      double Dl = j == 0 ? 1 : D, Dr = j == L - 1 ? 1 : D;
      double m = (double)rprev * D, n = b * Dr;
      f += 2.0 * rprev * Dl * p * b * a;            // S1
      f += 2.0 * rprev * D * b * Dr * Dl * p;       // X
      double kq = std::min(m, n);
      f += 2.0 * m * n * kq - (2.0 / 3.0) * kq * kq * kq;  // Householder R
      rprev = st.r[j];
    }
    int cn = 1;
    for (int j = L - 1; j >= 0; --j) {
      double a = st.ia[j], p = st.ip[j], b = st.ib[j];
      double Dl = j == 0 ? 1 : D, Dr = j == L - 1 ? 1 : D;
      f += 2.0 * a * p * Dr * cn * b;               // S2
      f += 2.0 * a * Dl * D * cn * p * Dr;          // Y
      if (j == 0) break;
      double rr = st.r[j - 1], n = (double)D * cn, A = a * Dl, kk = st.oa[j];
      f += 2.0 * rr * n * A;                        // X_j = R Y
      if (rr > n) f += 2.0 * rr * n * n - (2.0 / 3.0) * n * n * n;
      double q = std::min(rr, n);
      f += 4.0 * n * q * q - (4.0 / 3.0) * q * q * q;  // bidiagonalisation
      f += kk * 80.0 * q;                           // inverse iteration
      f += 2.0 * kk * kk * q;                       // Gram-Schmidt
      f += kk * (4.0 * n * q - 2.0 * q * q);        // back-transformation
      f += 2.0 * A * kk * n;                        // C_j
      cn = st.oa[j];
    }
    return f;
  };
  double envs = 0.0;  // one direction: L-1 compressions
  for (int t = 0; t < L - 1; ++t) envs += compress_flops(steps[t]);
  auto ud = [&](int row, int j, int which) -> double {  // U_row dims
    if (row < 0) return 1.0;
    return which == 0 ? steps[row].oa[j] : steps[row].ob[j];
  };
  auto dd = [&](int row, int j, int which) -> double {  // Dn_row dims
    if (row >= L) return 1.0;
    int t = L - 1 - row;
    return which == 0 ? steps[t].oa[j] : steps[t].ob[j];
  };
  // strips: evaluation (envs, ratios, B tensors) and sweep (right envs, left
  // advance, num/den of the proposals), antiparallel pairs at half filling
  double eval_strips = 0.0, sweep_strips = 0.0;
  for (int i = 0; i < L; ++i) {
    double pu = i == 0 ? 1 : D, pd = i == L - 1 ? 1 : D;
    for (int j = 0; j < L; ++j) {
      double Dl = j == 0 ? 1 : D, Dr = j == L - 1 ? 1 : D;
      double au = ud(i - 1, j, 0), bu = ud(i - 1, j, 1), ad = dd(i + 1, j, 0), bd = dd(i + 1, j, 1);
      double step1 = 2 * Dl * ad * pu * bu * au + 2 * ad * bu * Dr * pd * Dl * pu + 2 * bu * Dr * bd * ad * pd;
      eval_strips += 2 * step1;                                        // left + right envs
      eval_strips += 2 * Dl * ad * pu * bu * au + 2 * bu * Dr * ad * pd * bd + 2 * Dl * Dr * pu * pd * ad * bu;  // B
      sweep_strips += 2 * step1;                                       // right env + left advance
      if (j + 1 < L) {
        eval_strips += 0.5 * 2 * step1;                                // horizontal ratio (2 steps)
        sweep_strips += 0.5 * 3 * step1;  // num (2 steps) + den (2, the first is the left advance)
      }
      if (i + 1 < L) {
        double pd2 = i + 1 == L - 1 ? 1 : D;
        double ad2 = dd(i + 2, j, 0), bd2 = dd(i + 2, j, 1);
        double s2 = 2 * Dl * Dl * ad2 * pu * bu * au + 2 * Dl * ad2 * bu * Dr * D * Dl * pu +
                    2 * ad2 * bu * Dr * Dr * pd2 * Dl * D + 2 * bu * Dr * Dr * bd2 * ad2 * pd2;
        eval_strips += 2 * s2;                                         // left + right envs
        eval_strips += 0.5 * s2 + (j + 1 < L ? 0.5 * 2 * 2 * s2 : 0);  // v, d, a ratios
        sweep_strips += 2 * s2 + 0.5 * s2;  // right env, left advance (= den), num
      }
    }
  }
  if (what == 0) return 2.0 * envs + eval_strips;
  if (what == 1) return 2.0 * envs + sweep_strips;
  return 3.0 * envs + eval_strips + sweep_strips;  // the fused step reuses Dn
}

}  // extern "C"
