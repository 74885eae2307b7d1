// Kernels of order 9 (see enomr_orders.cuh).
#define ENOMR_R 9
#include "enomr_orders.cuh"
