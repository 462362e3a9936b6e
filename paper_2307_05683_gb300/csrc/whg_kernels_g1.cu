// whg_kernels_g1.cu -- kernel instances for 1 lane(s) per system.
#include "whg_device.cuh"

WHG_DEFINE_KERNEL_TABLE(1)
