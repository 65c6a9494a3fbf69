// Single-pass aggregation kernels for the paper's colour power bases.
#include "hgf_onepass.cuh"

HGF_INSTANTIATE_ONEPASS(hgf::B_RGB_POW2)
HGF_INSTANTIATE_ONEPASS(hgf::B_RGB_POW3)
