// tll_kern_k29.cu -- likelihood kernels with the compiled convolution
// for PSF sides 29, 31 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 29: return single_for<29>(sub);
        case 31: return single_for<31>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 29: return multi_for<29>(sub);
        case 31: return multi_for<31>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 29: return nc_for<29>(sub);
        case 31: return nc_for<31>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 29: return nc_multi_for<29>(sub);
        case 31: return nc_multi_for<31>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k29 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
