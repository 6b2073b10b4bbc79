// stage_f32.cu -- FP32 instances of the stage kernel (one per count of stage
// derivatives and demag sources read, last stage or not) and the controller
// kernel; a translation unit of its own so that it compiles in parallel.
#include "stage_tab.cuh"

const void *mmxk_stage_tab_f32(int nf, int nh, bool last, bool stage0) { return stage_tab<float>(nf, nh, last, stage0); }
const void *mmxk_control_f32() { return (const void *)k_control<float>; }
