// D2Q9 back end of liblbm.
#include "backend.cuh"

template struct lbm::Backend<9>;
