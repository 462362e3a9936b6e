// whg_kernels_g2.cu -- kernel instances for 2 lane(s) per system.
#include "whg_device.cuh"

WHG_DEFINE_KERNEL_TABLE(2)
