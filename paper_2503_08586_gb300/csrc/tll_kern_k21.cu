// tll_kern_k21.cu -- likelihood kernels with the compiled convolution
// for PSF sides 21, 23 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 21: return single_for<21>(sub);
        case 23: return single_for<23>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 21: return multi_for<21>(sub);
        case 23: return multi_for<23>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 21: return nc_for<21>(sub);
        case 23: return nc_for<23>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 21: return nc_multi_for<21>(sub);
        case 23: return nc_multi_for<23>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k21 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
