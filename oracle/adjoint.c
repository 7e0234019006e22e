/* oracle/adjoint.c -- TEST INFRASTRUCTURE ONLY (filled in with the adjoint). */
