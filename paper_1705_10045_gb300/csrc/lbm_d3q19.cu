// D3Q19 back end of liblbm.
#include "backend.cuh"

template struct lbm::Backend<19>;
