// fft_fused_f64.cu -- FP64 instances of the x passes and the fused y-z pass.
#include "kernels_impl.cuh"

const void *mmxk_tab_fused_f32(int kind, int L);

const void *mmxk_tab_fused(int kind, bool f64, int L)
{
    if (!f64) return mmxk_tab_fused_f32(kind, L);
    switch (kind) {
    case K_XF: return xf_fn<double>(L);
    case K_XI: return xi_fn<double>(L);
    case K_YZ: return yz_fn<double>(L);
    }
    return nullptr;
}
