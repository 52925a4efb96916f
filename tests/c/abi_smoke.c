/* Plain C11 client of the C ABI: compiles against include/tgp.h with no C++
 * and no CUDA headers, links libtgp.so, and exercises only the host-side
 * paths (status strings, version, argument checks that return before any
 * device work), so it runs without a GPU.  Prints "ok" on success. */
#include <stdio.h>
#include <string.h>

#include "tgp.h"

#define CHECK(cond)                                              \
  do {                                                           \
    if (!(cond)) {                                               \
      fprintf(stderr, "check failed: %s (line %d)\n", #cond, __LINE__); \
      return 1;                                                  \
    }                                                            \
  } while (0)

int main(void) {
  CHECK(strcmp(tgp_status_string(TGP_OK), "TGP_OK") == 0);
  CHECK(strstr(tgp_version(), "sm_103a") != NULL);

  /* population with null arrays but pop > 0: rejected on the host */
  tgp_population bad = {NULL, NULL, NULL, 4, 8, 8};
  tgp_data data = {NULL, 0, 1, 1};
  CHECK(tgp_fitness_mse(&bad, &data, NULL, 1, NULL, NULL, NULL, 0, NULL) == TGP_ERR_INVALID_ARG);

  /* max_len beyond the library limit */
  tgp_population wide = {NULL, NULL, NULL, 0, TGP_MAX_LEN + 1, TGP_MAX_LEN + 1};
  CHECK(tgp_eval_forward(&wide, &data, 1, NULL, NULL, NULL, 0, NULL) == TGP_ERR_INVALID_ARG);

  /* genetic operators: bad mode, bad size limit, nothing to do */
  tgp_population empty = {NULL, NULL, NULL, 0, 8, 8};
  CHECK(tgp_subtree_exchange(&empty, &empty, NULL, NULL, NULL, NULL, NULL, 0u, 1, 7, 8, NULL, NULL,
                             NULL, 8, NULL, NULL) == TGP_ERR_INVALID_ARG);
  CHECK(tgp_subtree_exchange(&empty, &empty, NULL, NULL, NULL, NULL, NULL, 0u, 1, TGP_PICK_RANDOM, 0,
                             NULL, NULL, NULL, 8, NULL, NULL) == TGP_ERR_INVALID_ARG);
  CHECK(tgp_subtree_exchange(&empty, &empty, NULL, NULL, NULL, NULL, NULL, 0u, 0, TGP_PICK_HOIST, 8,
                             NULL, NULL, NULL, 8, NULL, NULL) == TGP_OK);
  CHECK(tgp_tournament_select(NULL, 1, 10, NULL, 0, 20, 1, NULL, NULL) == TGP_OK);
  CHECK(tgp_tournament_select(NULL, 1, 10, NULL, 5, 20, 1, NULL, NULL) == TGP_ERR_INVALID_ARG);
  CHECK(tgp_accuracy_from_outputs(NULL, 0, 3, 10, NULL, NULL, NULL, NULL) == TGP_OK);

  /* batch plan: argument checks and the host-only autotune cache lookup */
  tgp_batch_plan_t* plan = NULL;
  CHECK(tgp_batch_plan(NULL, 1, NULL, &plan) == TGP_ERR_INVALID_ARG && plan == NULL);
  CHECK(tgp_batch_plan_workspace_size(NULL) == 0);
  CHECK(tgp_batch_run(NULL, NULL, 0, NULL) == TGP_ERR_INVALID_ARG);
  tgp_batch_free(NULL);
  {
    const char* path = "abi_smoke_tune.txt";
    FILE* f = fopen(path, "w");
    CHECK(f != NULL);
    fprintf(f, "# comment\n");
    fprintf(f, "GPU_X|P13_D17_F16_O1_L8 trees_per_block=8 points_per_tile=512 tiles_per_item=2 "
               "points_per_lane=8 ms=1.5\n");
    fprintf(f, "GPU_X|P13_D17_F16_O1_L8 trees_per_block=28 points_per_tile=1024 tiles_per_item=0 "
               "points_per_lane=8 cta_width=2\n");
    fprintf(f, "GPU_X|P11_D11_F4_O1_L6 trees_per_block=8 cta_width=3\n");
    fprintf(f, "GPU_X|P10_D10_F4_O1_L6 trees_per_block=x\n");
    fclose(f);
    tgp_config c;
    memset(&c, 0, sizeof c);
    CHECK(tgp_tune_cache_lookup(path, "GPU_X|P13_D17_F16_O1_L8", &c) == TGP_OK);
    CHECK(c.trees_per_block == 28 && c.points_per_tile == 1024 && c.tiles_per_item == 0 &&
          c.points_per_lane == 8 && c.cta_width == 2 && c.flags == 0);
    CHECK(tgp_tune_cache_lookup(path, "GPU_X|P11_D11_F4_O1_L6", &c) == TGP_ERR_INVALID_ARG);
    CHECK(tgp_tune_cache_lookup(path, "GPU_X|P10_D10_F4_O1_L6", &c) == TGP_ERR_INVALID_ARG);
    CHECK(tgp_tune_cache_lookup(path, "GPU_Y|P13_D17_F16_O1_L8", &c) == TGP_ERR_INVALID_ARG);
    CHECK(tgp_tune_cache_lookup("no_such_file.txt", "GPU_X|P13_D17_F16_O1_L8", &c) ==
          TGP_ERR_INVALID_ARG);
    remove(path);
  }
  printf("ok\n");
  return 0;
}
