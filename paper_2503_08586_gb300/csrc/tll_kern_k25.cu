// tll_kern_k25.cu -- likelihood kernels with the compiled convolution
// for PSF sides 25, 27 (one translation unit per pair, compiled in parallel).
#include "tll_multi.cuh"

namespace tll {
namespace {

SingleKernel single_k(int sub, int K, bool write)
{
    if (write) return nullptr;
    switch (K) {
        case 25: return single_for<25>(sub);
        case 27: return single_for<27>(sub);
    }
    return nullptr;
}

MultiKernel multi_k(int sub, int K)
{
    switch (K) {
        case 25: return multi_for<25>(sub);
        case 27: return multi_for<27>(sub);
    }
    return nullptr;
}

NcKernel nc_k(int sub, int K)
{
    switch (K) {
        case 25: return nc_for<25>(sub);
        case 27: return nc_for<27>(sub);
    }
    return nullptr;
}

MultiKernel nc_multi_k(int sub, int K)
{
    switch (K) {
        case 25: return nc_multi_for<25>(sub);
        case 27: return nc_multi_for<27>(sub);
    }
    return nullptr;
}

}  // namespace

extern const KernelSet kernel_set_k25 = {single_k, multi_k, nc_k, nc_multi_k};

}  // namespace tll
