// Kernels of order 7 (see enomr_orders.cuh).
#define ENOMR_R 7
#include "enomr_orders.cuh"
