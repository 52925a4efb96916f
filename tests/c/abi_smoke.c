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
  printf("ok\n");
  return 0;
}
