/* A C-only caller of libcamelot: creates a predictor from parameters in a
 * file, builds the allocator's table from it (camelot_profile_predict) and
 * solves Eq. 1 (camelot_allocate), printing the allocation.  Used by the GPU
 * tests to show that allocation from the predictor needs no Python.
 *
 * usage: alloc_from_predictor <params.f32> <norm.f32> <total_sms>
 *   params.f32: CAMELOT_PRED_PARAMS floats; norm.f32: 12 means then 12 inverse
 *   standard deviations.  Output: "instances n0 n1 quota q0 q1 batch b objective x". */
#include <stdio.h>
#include <stdlib.h>

#include "camelot.h"

static int read_f32(const char* path, float* out, size_t n) {
    FILE* f = fopen(path, "rb");
    if (!f) return -1;
    size_t got = fread(out, sizeof(float), n, f);
    fclose(f);
    return got == n ? 0 : -1;
}

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    static float params[CAMELOT_PRED_PARAMS];
    float norm[2 * CAMELOT_PRED_FEATURES];
    if (read_f32(argv[1], params, CAMELOT_PRED_PARAMS) || read_f32(argv[2], norm, 2 * CAMELOT_PRED_FEATURES))
        return 3;
    const int total = atoi(argv[3]);
    camelot_predictor* p = NULL;
    if (camelot_predictor_create(params, &p) != CAMELOT_OK) return 4;
    if (camelot_predictor_set_norm(p, norm, norm + CAMELOT_PRED_FEATURES) != CAMELOT_OK) return 5;
    /* the two stages of the plain 2-stage pipeline: normalise, MLP 12288-512-256-10 */
    const double macs = 12288.0 * 512 + 512.0 * 256 + 256.0 * 10;
    camelot_stage_cost costs[2] = {{1, 0, 2.0 * 12288, 0.0, 12288.0 + 49152.0, 64e6},
                                   {2, 0, 2.0 * macs, 4.0 * macs, 49152.0 + 8.0, 64e6}};
    const int32_t batches[4] = {8, 16, 32, 64};
    const int L = total / 8;
    double* thr = malloc(sizeof(double) * 4 * 2 * L);
    double* bw = malloc(sizeof(double) * 4 * 2 * L);
    double* dur = malloc(sizeof(double) * 4 * 2 * L);
    double mem[8];
    if (camelot_profile_predict(p, costs, 2, batches, 4, 8, L, 0, 0.0, thr, bw, dur, mem) != CAMELOT_OK) {
        fprintf(stderr, "%s\n", camelot_last_error());
        return 6;
    }
    camelot_profile prof = {2, L, 4, 8, batches, thr, bw, dur, mem};
    camelot_constraints c = {total, total / 8, 1e9, 1e12, 20e-3, 0.0, CAMELOT_SOLVER_EXHAUSTIVE, 0, 0.0, 0.0, 0};
    camelot_alloc a;
    double obj = 0.0;
    if (camelot_allocate(&prof, CAMELOT_POLICY_MAX_PEAK, &c, &a, &obj) != CAMELOT_OK) {
        fprintf(stderr, "%s\n", camelot_last_error());
        return 7;
    }
    printf("instances %d %d quota %d %d batch %d objective %.17g\n", a.instances[0], a.instances[1], a.sm_quota[0],
           a.sm_quota[1], a.batch, obj);
    camelot_predictor_destroy(p);
    free(thr);
    free(bw);
    free(dur);
    return 0;
}
