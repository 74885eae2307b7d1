// Kernels of order 17 (see enomr_orders.cuh).
#define ENOMR_R 17
#include "enomr_orders.cuh"
