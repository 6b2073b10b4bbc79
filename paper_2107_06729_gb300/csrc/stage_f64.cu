// stage_f64.cu -- FP64 instances of the stage kernel and the controller kernel.
#include "stage_tab.cuh"

const void *mmxk_stage_tab_f64(int nf, int nh, bool last, bool stage0) { return stage_tab<double>(nf, nh, last, stage0); }
const void *mmxk_control_f64() { return (const void *)k_control<double>; }
