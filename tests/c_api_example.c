/* The library from C: build a table of two patterns, search a host text with
 * rk_search, print the sorted (pattern id, offset) list, one match per line.
 * tests/test_abi.py compiles and links it; tests/test_gpu_search.py runs it
 * on a GPU and checks the output. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "rk.h"

int main(void) {
    const char *text = "xxGATTACAxACGTxxGATTACA";
    const char *patterns = "GATTACA" "ACGT"; /* concatenated; ids 0 and 1 */
    const uint32_t lens[2] = {7, 4};
    rk_table *t = NULL;
    int rc = rk_build((const uint8_t *)patterns, lens, 2, NULL, &t);
    if (rc != RK_OK) {
        fprintf(stderr, "rk_build: %s\n", rk_strerror(rc));
        return 1;
    }
    uint64_t keys[16], n = 0;
    rc = rk_search(t, (const uint8_t *)text, strlen(text), keys, 16, &n);
    if (rc != RK_OK) {
        fprintf(stderr, "rk_search: %s\n", rk_strerror(rc));
        rk_destroy(t);
        return 1;
    }
    for (uint64_t i = 0; i < n; ++i)
        printf("%u %llu\n", RK_KEY_ID(keys[i]), (unsigned long long)RK_KEY_OFFSET(keys[i]));
    rk_destroy(t);
    return 0;
}
