// Launchers of the kernel families a counting build of the emulation leaves
// out (it compiles the float-float fused kernel's unit only, so that the
// phase counters it reads are the ones its functions update): each returns
// an error.
#include "cuda_runtime.h"
#include "peps_args.h"
#include "peps_launch.h"

cudaError_t peps_launch_eval_f64(const EvalArgs<double>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_eval_ff(const EvalArgs<ff>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_eval_f32(const EvalArgs<float>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_sample_f64(const SampleArgs<double>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_sample_ff(const SampleArgs<ff>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_sample_f32(const SampleArgs<float>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_vmc_f64(const EvalArgs<double>&, const SampleArgs<double>&, int,
                                cudaStream_t) { return 1; }
cudaError_t peps_launch_vmc_f32(const EvalArgs<float>&, const SampleArgs<float>&, int,
                                cudaStream_t) { return 1; }
cudaError_t peps_launch_corr_f64(const CorrArgs<double>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_corr_ff(const CorrArgs<ff>&, int, cudaStream_t) { return 1; }
cudaError_t peps_launch_multi_f64(const MultiJobDev<double>*, int, int64_t, unsigned long long*,
                                  double*, double*, int64_t, int64_t, int*, int, cudaStream_t) {
  return 1;
}
cudaError_t peps_launch_multi_ff(const MultiJobDev<ff>*, int, int64_t, unsigned long long*, ff*,
                                 double*, int64_t, int64_t, int*, int, cudaStream_t) {
  return 1;
}
int peps_phase_read_f64(unsigned long long*, int) { return 0; }
int peps_phase_read_f32(unsigned long long*, int) { return 0; }
