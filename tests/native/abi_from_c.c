/*
 * Test driver for tests/test_abi.py: include/tc.h compiled as plain C11 and linked against
 * libtcgb300.so, calling the entry points that return before any device work (status strings,
 * version, default options, argument checks).  Exits 0 when every result is the documented one.
 */
#include <stdio.h>
#include <string.h>

#include "tc.h"

#define EXPECT(c)                                                    \
    do {                                                             \
        if (!(c)) {                                                  \
            fprintf(stderr, "failed: %s (line %d)\n", #c, __LINE__); \
            return 1;                                                \
        }                                                            \
    } while (0)

int main(void) {
    EXPECT(strcmp(tc_status_str(TC_OK), "ok") == 0);
    EXPECT(tc_status_str((tc_status)99) != NULL);
    EXPECT(strstr(tc_version(), "sm_103a") != NULL);
    tc_options o;
    tc_options_default(&o);
    EXPECT(o.piece == 2048 && o.small_max == 64 && o.static_percent == 50 && o.cost_model == TC_COST_EDGE);
    tc_graph_t g = NULL;
    EXPECT(tc_build(NULL, NULL, -1, 10, NULL, NULL, &g) == TC_ERR_INVALID_ARG && g == NULL);
    EXPECT(tc_build_pairs(NULL, 3, 10, NULL, NULL, &g) == TC_ERR_INVALID_ARG);
    o.piece = 1000;
    EXPECT(tc_build(NULL, NULL, 0, 10, &o, NULL, &g) == TC_ERR_INVALID_ARG);
    uint64_t t = 0;
    EXPECT(tc_count(NULL, NULL, &t) == TC_ERR_INVALID_ARG);
    EXPECT(tc_count_graphs(NULL, -1, NULL, &t) == TC_ERR_INVALID_ARG);
    int64_t off[3] = {0, 0, 0};
    int32_t cuts[3] = {0, 3, 2};  /* decreasing: refused */
    EXPECT(tc_count_surrogate(off, NULL, 2, 0, cuts, 2, 0, 2, NULL, NULL, NULL, &t, NULL) == TC_ERR_INVALID_ARG);
    int32_t P = 0;
    EXPECT(tc_surrogate_plan(off, NULL, 2, 0, TC_FN_LIST + 1, 1, 0, 1, NULL, cuts, &P) == TC_ERR_INVALID_ARG);
    tc_free(NULL);
    tc_batch_free(NULL);
    tc_server_destroy(NULL);
    printf("abi from C: ok\n");
    return 0;
}
