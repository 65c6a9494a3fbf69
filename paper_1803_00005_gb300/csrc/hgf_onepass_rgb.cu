// Single-pass aggregation kernels for the RGB bases with n <= 9.
#include "hgf_onepass.cuh"

HGF_INSTANTIATE_ONEPASS(hgf::B_RGB_MONO1)
HGF_INSTANTIATE_ONEPASS(hgf::B_RGB_MONO2)
