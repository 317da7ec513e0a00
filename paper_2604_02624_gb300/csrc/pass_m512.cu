// Row and column pass kernels for padded size M = 512 = 16 x 32, 16 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(512, 16, 32, 16, 8)
