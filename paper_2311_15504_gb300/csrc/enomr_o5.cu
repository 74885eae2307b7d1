// Kernels of order 5 (see enomr_orders.cuh).
#define ENOMR_R 5
#include "enomr_orders.cuh"
