// whg_kernels_g8.cu -- kernel instances for 8 lane(s) per system.
#include "whg_device.cuh"

WHG_DEFINE_KERNEL_TABLE(8)
