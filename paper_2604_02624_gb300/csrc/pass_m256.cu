// Row and column pass kernels for padded size M = 256 = 16 x 16, 16 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(256, 16, 16, 16, 16)
