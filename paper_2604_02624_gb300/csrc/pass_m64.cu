// Row and column pass kernels for padded size M = 64 = 8 x 8, 8 threads per line.
#include "dos_pass_bulk.cuh"
DOS_DEFINE_PASS_OPS(64, 8, 8, 8, 16)
