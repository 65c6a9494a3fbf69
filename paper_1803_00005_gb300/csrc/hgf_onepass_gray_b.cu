// Single-pass aggregation kernels for gray powers I..I^d, d = 6..9.
#include "hgf_onepass.cuh"

HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY6)
HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY7)
HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY8)
HGF_INSTANTIATE_ONEPASS(hgf::B_GRAY9)
