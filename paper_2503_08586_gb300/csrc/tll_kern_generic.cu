// tll_kern_generic.cu -- likelihood kernels with the generic (runtime PSF
// side) convolution, including the write-out variants of the model-image
// entry points.
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (K != 0) return nullptr;
    switch (sub_class(sub)) {
        case 4: return write ? k_loglike<4, 0, true> : k_loglike<4, 0, false>;
        case 5: return write ? k_loglike<5, 0, true> : k_loglike<5, 0, false>;
        default: return write ? k_loglike<0, 0, true> : k_loglike<0, 0, false>;
    }
}

MultiKernel multi_k(int sub, int K)
{
    return K == 0 ? multi_for<0>(sub) : nullptr;
}

NcKernel nc_k(int sub, int K)
{
    return K == 0 ? nc_for<0>(sub) : nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    return K == 0 ? nc_multi_for<0>(sub) : nullptr;
}

}  // namespace

extern const KernelSet kernel_set_generic = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
