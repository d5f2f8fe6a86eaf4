// tll_kern_k13.cu -- likelihood kernels with the compiled convolution
// for PSF sides 13, 15 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 13: return single_for<13>(sub);
        case 15: return single_for<15>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 13: return multi_for<13>(sub);
        case 15: return multi_for<15>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 13: return nc_for<13>(sub);
        case 15: return nc_for<15>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 13: return nc_multi_for<13>(sub);
        case 15: return nc_multi_for<15>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k13 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
