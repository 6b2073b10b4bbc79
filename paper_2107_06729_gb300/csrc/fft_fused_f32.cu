// fft_fused_f32.cu -- FP32 instances of the x passes and the fused y-z pass.
#include "kernels_impl.cuh"

const void *mmxk_tab_fused_f32(int kind, int L)
{
    switch (kind) {
    case K_XF: return xf_fn<float>(L);
    case K_XI: return xi_fn<float>(L);
    case K_YZ: return yz_fn<float>(L);
    }
    return nullptr;
}
