/* Internal helpers of the FP64 oracle (test infrastructure only). */
#ifndef SWEEP_ORACLE_INTERNAL_H
#define SWEEP_ORACLE_INTERNAL_H
#ifndef _GNU_SOURCE
#define _GNU_SOURCE
#endif
#include "oracle.h"

#include <stddef.h>

#define ORC_EINVAL (-1)
#define ORC_EBOUNDS (-3)

extern const double ORC_C2[5];
extern const double ORC_C1[5];
extern const double ORC_S1;
extern const double ORC_S2;

/* edge-replicated (or copied, if already padded) model, caller frees */
double* orc_pad_model(const oracle_problem* p, const double* model, int npar);
int orc_check(const oracle_problem* p, const int32_t* src, const int32_t* rec);

#endif
