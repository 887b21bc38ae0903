/* A C99 caller of the C ABI (include/countgauss.h), built and run by test_abi.py without a
 * GPU: plans, options, workspace queries and the host-side argument checks, which return
 * before any CUDA call.  Prints "ok" and exits 0 when every check holds. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "countgauss.h"

#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            printf("failed at line %d: %s\n", __LINE__, #cond);     \
            return 1;                                                 \
        }                                                             \
    } while (0)

int main(void) {
    cg_plan *plan = NULL;
    CHECK(cg_plan_create(1000, 16, 8, 256, 42, &plan) == CG_OK && plan != NULL);
    cg_plan *bad = NULL;
    CHECK(cg_plan_create(-1, 16, 8, 256, 42, &bad) == CG_ERR_INVALID_ARG && bad == NULL);
    CHECK(cg_plan_create(1000, 0, 8, 256, 42, &bad) == CG_ERR_INVALID_ARG && bad == NULL);

    int64_t v = -1;
    CHECK(cg_plan_set_option(plan, CG_OPT_PRECISION, CG_PREC_BF16X3) == CG_OK);
    CHECK(cg_plan_get_option(plan, CG_OPT_PRECISION, &v) == CG_OK && v == CG_PREC_BF16X3);
    CHECK(cg_plan_set_option(plan, CG_OPT_PRECISION, 99) == CG_ERR_INVALID_ARG);
    CHECK(cg_plan_set_option(plan, CG_OPT_ROW_OFFSET, (int64_t)1 << 40) == CG_OK);
    CHECK(cg_plan_get_option(plan, CG_OPT_ROW_OFFSET, &v) == CG_OK && v == (int64_t)1 << 40);

    size_t bytes = 0;
    CHECK(cg_workspace_size(plan, CG_OP_APPLY_CSR, 5000, &bytes) == CG_OK);
    CHECK(bytes >= 256 + (size_t)256 * 16 * sizeof(float) && bytes % 256 == 0);
    CHECK(cg_workspace_size(plan, CG_OP_SKETCH_I64, (int64_t)1 << 35, &bytes) == CG_OK && bytes == 256);
    CHECK(cg_workspace_size(plan, 77, 0, &bytes) == CG_ERR_INVALID_ARG);

    /* argument checks that return before any CUDA call (the pointers are never used) */
    void *fake = (void *)(uintptr_t)(1u << 20);
    float *Y = (float *)fake;
    CHECK(cg_apply_csr(plan, (const int32_t *)fake, (const int32_t *)fake, (const float *)fake, -1, Y, fake,
                       1u << 30, NULL) == CG_ERR_INVALID_ARG);
    CHECK(cg_apply_csr(plan, (const int32_t *)fake, (const int32_t *)fake, (const float *)fake, 10, Y, fake, 16,
                       NULL) == CG_ERR_WORKSPACE);
    CHECK(cg_apply_csr_i64(plan, (const int64_t *)((char *)fake + 4), (const int32_t *)fake, (const float *)fake, 10,
                           Y, fake, 1u << 30, NULL) == CG_ERR_INVALID_ARG);
    CHECK(cg_plan_set_option(plan, CG_OPT_DETERMINISTIC, 1) == CG_OK);
    CHECK(cg_apply_right_csr(plan, (const int32_t *)fake, (const int32_t *)fake, (const float *)fake, 10, Y, fake,
                             1u << 30, NULL) == CG_ERR_UNSUPPORTED);

    for (int s = CG_OK; s <= CG_ERR_NO_DEVICE; ++s) {
        const char *str = cg_status_string((cg_status)s);
        CHECK(str != NULL && strlen(str) > 0);
    }
    CHECK(cg_plan_destroy(plan) == CG_OK);
    printf("ok\n");
    return 0;
}
