// tll_kern_k09.cu -- likelihood kernels with the compiled convolution
// for PSF sides 9, 11 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 9: return single_for<9>(sub);
        case 11: return single_for<11>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 9: return multi_for<9>(sub);
        case 11: return multi_for<11>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 9: return nc_for<9>(sub);
        case 11: return nc_for<11>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 9: return nc_multi_for<9>(sub);
        case 11: return nc_multi_for<11>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k09 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
