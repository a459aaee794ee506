/* A plain C99 caller of the C ABI (include/ctis.h), host-only entry points:
 * builds the work lists of a tiny plan with ctis_tables_inspect and reports
 * them, then checks the error path. Compiled and run by tests/test_abi.py. */
#include <stdio.h>
#include <string.h>

#include "ctis.h"

int main(void) {
    /* field stop 4 x 3, 2 wavelengths, 10 x 9 FPA; two nonzeros each */
    const int32_t ptr[3] = {0, 2, 4};
    const int32_t x[4] = {1, 2, 5, 6};
    const int32_t y[4] = {0, 0, 3, 4};
    const float v[4] = {0.5f, 0.25f, 1.0f, 0.75f};
    ctis_tables_info info;
    memset(&info, 0, sizeof info);
    info.struct_size = (int)sizeof info;
    int rc = ctis_tables_inspect(4, 3, 2, 10, 9, ptr, x, y, v, CTIS_F32, NULL, 1, 4, NULL, &info,
                                 NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    if (rc != CTIS_OK) {
        printf("inspect failed: %s (%s)\n", ctis_status_string(rc), ctis_last_error());
        return 1;
    }
    printf("clusters %lld k %lld tiles %lld tasks %lld\n", (long long)info.clusters,
           (long long)info.cluster_k, (long long)info.tiles, (long long)info.tasks);
    /* a shifted copy past the FPA under the default (reject) boundary */
    const int32_t xbad[4] = {1, 2, 7, 6};
    rc = ctis_tables_inspect(4, 3, 2, 10, 9, ptr, xbad, y, v, CTIS_F32, NULL, 1, 4, NULL, &info,
                             NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    printf("reject %s\n", ctis_status_string(rc));
    return rc == CTIS_ERR_OUT_OF_BOUNDS ? 0 : 1;
}
