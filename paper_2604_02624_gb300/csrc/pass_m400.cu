// Row and column pass kernels for padded size M = 400 = 20 x 20, 20 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(400, 20, 20, 20, 8)
