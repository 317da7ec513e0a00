// Row and column pass kernels for padded size M = 128 = 8 x 16, 8 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(128, 8, 16, 8, 16)
