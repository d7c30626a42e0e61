// Definitions the plan builder links against from other translation units
// of the library, replaced for a host-only build of plan.cu (no device
// calls are made by the list builder under test).
#include "prop_internal.cuh"
namespace prop {
prop_status fail(prop_status s, const std::string&) { return s; }
prop_status cuda_fail(cudaError_t, const char*) { return PROP_ERR_CUDA; }
void set_error(const std::string&) {}
void fft_make_maps(Plan&) {}
cudaError_t fft_configure(int) { return cudaSuccess; }
cudaError_t nufft_configure(int) { return cudaSuccess; }
int interp_buffers(const Plan&) { return 1; }
}  // namespace prop
