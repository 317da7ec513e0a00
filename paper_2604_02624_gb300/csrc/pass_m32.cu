// Row and column pass kernels for padded size M = 32 = 4 x 8, 4 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(32, 4, 8, 4, 16)
