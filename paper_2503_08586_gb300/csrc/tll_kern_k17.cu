// tll_kern_k17.cu -- likelihood kernels with the compiled convolution
// for PSF sides 17, 19 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 17: return single_for<17>(sub);
        case 19: return single_for<19>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 17: return multi_for<17>(sub);
        case 19: return multi_for<19>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 17: return nc_for<17>(sub);
        case 19: return nc_for<19>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 17: return nc_multi_for<17>(sub);
        case 19: return nc_multi_for<19>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k17 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
