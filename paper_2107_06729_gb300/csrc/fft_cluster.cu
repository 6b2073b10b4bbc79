// fft_cluster.cu -- instances of the cluster-fused y-z pass (YZC, FP32).
#include "kernels_impl.cuh"

const void *mmxk_yzc_kernel(int Py, int Pz)
{
    switch (Py) {
    case 128: return yzc_fn_z<128>(Pz);
    case 256: return yzc_fn_z<256>(Pz);
    case 512: return yzc_fn_z<512>(Pz);
    case 1024: return yzc_fn_z<1024>(Pz);
    }
    return nullptr;
}
