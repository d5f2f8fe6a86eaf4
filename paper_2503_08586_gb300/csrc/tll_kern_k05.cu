// tll_kern_k05.cu -- likelihood kernels with the compiled convolution
// for PSF sides 5, 7 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 5: return single_for<5>(sub);
        case 7: return single_for<7>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 5: return multi_for<5>(sub);
        case 7: return multi_for<7>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 5: return nc_for<5>(sub);
        case 7: return nc_for<7>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 5: return nc_multi_for<5>(sub);
        case 7: return nc_multi_for<7>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k05 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
