// tll_kern_k01.cu -- likelihood kernels with the compiled convolution
// for PSF sides 1, 3 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 1: return single_for<1>(sub);
        case 3: return single_for<3>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 1: return multi_for<1>(sub);
        case 3: return multi_for<3>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 1: return nc_for<1>(sub);
        case 3: return nc_for<3>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 1: return nc_multi_for<1>(sub);
        case 3: return nc_multi_for<3>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k01 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
