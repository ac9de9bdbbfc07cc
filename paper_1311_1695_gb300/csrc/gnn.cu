// GNN kernels (warm start): filled in below.
#include "common.cuh"
