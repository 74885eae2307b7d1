// Kernels of order 11 (see enomr_orders.cuh).
#define ENOMR_R 11
#include "enomr_orders.cuh"
