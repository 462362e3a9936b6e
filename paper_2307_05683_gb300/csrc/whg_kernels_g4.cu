// whg_kernels_g4.cu -- kernel instances for 4 lane(s) per system.
#include "whg_device.cuh"

WHG_DEFINE_KERNEL_TABLE(4)
