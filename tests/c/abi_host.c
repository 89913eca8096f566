/* A plain C99 client of liblbm: includes the public header, links the
 * library and calls the entry points that need no GPU.  tests/test_c_abi.py
 * compiles and runs it and checks what it prints. */
#include <stdio.h>
#include <string.h>

#include "lbm.h"

int main(void) {
    lbm_params p;
    lbm_default_params(&p);
    printf("sizeof_params %zu\n", sizeof(lbm_params));
    printf("sizeof_slab %zu\n", sizeof(lbm_slab));
    printf("defaults %d %d %d %d %.17g %.17g %d\n", p.lattice, p.nx, p.ny, p.nz, p.kappa, p.A, p.storage);
    printf("codes %d %d %d %d %d %d %d\n", LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_UNSTABLE_PARAMS, LBM_ERR_OOM,
           LBM_ERR_CUDA, LBM_ERR_NONPHYSICAL, LBM_ERR_TIMEOUT);

    double rv = 0.0, rl = 0.0;
    int rc = lbm_coexistence(0.8, &rv, &rl);
    printf("coexistence %d %.12f %.12f\n", rc, rv, rl);
    printf("coexistence_bad %d\n", lbm_coexistence(1.5, &rv, &rl));

    p.lattice = LBM_D3Q19;
    p.nx = 16;
    p.ny = 12;
    p.nz = 40;
    p.wall = 1;
    p.T_fixed_lo = 1;
    p.T_lo = 0.9;
    lbm_slab s;
    rc = lbm_slab_plan(&p, 3, 1, &s);
    printf("slab %d %d %d %d %d %d %d %d %d\n", rc, s.first, s.own, s.lo, s.hi, s.below, s.above, s.p.nz,
           s.p.T_fixed_lo);
    rc = lbm_slab_plan(&p, 21, 0, &s);
    printf("slab_thin %d %s\n", rc, strlen(lbm_last_error()) > 0 ? "msg" : "nomsg");

    lbm_handle* h = NULL;
    p.tau = 0.5;
    rc = lbm_create(&p, &h);
    printf("create_bad %d %s\n", rc, h == NULL ? "null" : "set");
    printf("null_step %d\n", lbm_step(NULL, 1));
    printf("null_bytes %zu\n", lbm_state_bytes(NULL));
    lbm_destroy(NULL);
    lbm_slabs_destroy(NULL);
    return 0;
}
