// Row and column pass kernels for padded size M = 16 = 4 x 4, 4 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(16, 4, 4, 4, 16)
