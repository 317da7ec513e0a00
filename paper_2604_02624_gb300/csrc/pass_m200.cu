// Row and column pass kernels for padded size M = 200 = 10 x 20, 10 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(200, 10, 20, 10, 16)
