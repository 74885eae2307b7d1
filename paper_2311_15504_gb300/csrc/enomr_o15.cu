// Kernels of order 15 (see enomr_orders.cuh).
#define ENOMR_R 15
#include "enomr_orders.cuh"
