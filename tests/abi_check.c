/* Host program of tests/test_abi_cpu.py: include/gw.h compiled as strict C and linked against
 * libgw.so; calls the entry points that need no GPU and prints what they return. */
#include <stdio.h>

#include "gw.h"

int main(void)
{
    gw_ctx *ctx = NULL;
    printf("version %d\n", gw_version());
    printf("status0 %s\n", gw_status_str(GW_OK));
    printf("status5 %s\n", gw_status_str(GW_E_NUMERIC));
    printf("null_destroy %d\n", (int)gw_destroy(NULL));
    printf("null_create %d\n", (int)gw_create(NULL, 0, NULL));
    printf("null_eps_inv %d\n", (int)gw_eps_inv(NULL, GW_INV_CHOLESKY, NULL, NULL));
    (void)ctx;
    return 0;
}
