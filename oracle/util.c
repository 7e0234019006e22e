/* oracle/util.c -- TEST INFRASTRUCTURE ONLY: small helpers of the CPU oracle. */
#include <omp.h>

/* Number of OpenMP threads the oracle's parallel loops use. */
int oracle_threads(void) { return omp_get_max_threads(); }
