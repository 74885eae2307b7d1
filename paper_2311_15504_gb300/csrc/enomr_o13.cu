// Kernels of order 13 (see enomr_orders.cuh).
#define ENOMR_R 13
#include "enomr_orders.cuh"
