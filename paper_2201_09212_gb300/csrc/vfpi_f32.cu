// float instantiation of the V-FPI kernels and launchers.
#include <algorithm>

#include "vfpi_launch.cuh"

template struct vfpi::Launch<float>;
