/* A plain C99 consumer of the library: includes the public header, takes the
 * address of every entry point (so each must link), and makes the calls that
 * need no GPU.  Built and run by tests/test_abi.py. */
#include <stdio.h>
#include <string.h>

#include "jt.h"

typedef void (*any_fn)(void);

int main(void) {
  const any_fn entry[] = {
      (any_fn)jt_load_tree,        (any_fn)jt_set_evidence,       (any_fn)jt_set_evidence_dense,
      (any_fn)jt_propagate,        (any_fn)jt_profile_propagate,  (any_fn)jt_get_marginal,
      (any_fn)jt_log_evidence,     (any_fn)jt_get_marginals,      (any_fn)jt_get_log_evidence,
      (any_fn)jt_get_status,       (any_fn)jt_get_clique,         (any_fn)jt_get_clique_noalloc,
      (any_fn)jt_propagate_per_message, (any_fn)jt_init_from_cpts, (any_fn)jt_get_potential,
      (any_fn)jt_get_info,         (any_fn)jt_get_schedule,       (any_fn)jt_propagate_ctas,
      (any_fn)jt_get_kernel_span,  (any_fn)jt_free,               (any_fn)jt_strerror,
      (any_fn)jt_last_error,
  };
  size_t i;
  for (i = 0; i < sizeof(entry) / sizeof(entry[0]); ++i)
    if (!entry[i]) return 1;
  if (strcmp(jt_strerror(JT_OK), "ok") != 0) return 2;
  /* a malformed descriptor is rejected on the host, before any device work */
  {
    jt_tree t = 0;
    jt_status s = jt_load_tree(NULL, NULL, &t);
    if (s != JT_ERR_INVALID_ARG || t != NULL) return 3;
  }
  jt_free(NULL);
  printf("c-abi ok %u entry points\n", (unsigned)(sizeof(entry) / sizeof(entry[0])));
  return 0;
}
