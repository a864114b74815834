/* A plain C11 program that uses librdct through include/rdct.h only: the
 * header must compile as C, the library must link from C, and the calls that
 * need no GPU (version, status names, argument validation, which runs before
 * anything touches the device) must behave as the header states. */
#include <stdio.h>
#include <string.h>

#include "rdct.h"

int main(void) {
    char msg[256];
    printf("version %d\n", (int)rdct_version());
    printf("status2 %s\n", rdct_status_string(RDCT_ERR_SHAPE));
    /* width 12 is not a multiple of 8: RDCT_ERR_SHAPE, nothing launched */
    rdct_plane bad = {(const uint8_t *)16, 16, 12, 8};
    int32_t *Y = (int32_t *)16;
    rdct_status st = rdct_forward(&bad, Y, NULL);
    rdct_last_error(msg, sizeof msg);
    printf("forward %d %s\n", (int)st, strstr(msg, "multiples of 8") ? "detail-ok" : msg);
    /* r = 0 is out of range: RDCT_ERR_ARG */
    rdct_plane ok = {(const uint8_t *)16, 16, 16, 8};
    st = rdct_fused(&ok, 0, RDCT_KIND_RDCT, NULL, (double *)16, NULL, NULL);
    printf("fused %d\n", (int)st);
    /* a batch job with a bad plane names the job */
    rdct_job jobs[1];
    memset(jobs, 0, sizeof jobs);
    jobs[0].src = bad;
    jobs[0].r = 10;
    rdct_plan *plan = NULL;
    st = rdct_batch_plan_create(jobs, 1, 1, NULL, &plan);
    rdct_last_error(msg, sizeof msg);
    printf("plan %d %s %s\n", (int)st, plan == NULL ? "null" : "set", strstr(msg, "batch job 0") ? "named" : msg);
    return 0;
}
