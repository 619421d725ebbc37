// Optional subsystems attached to a context.
#include "cm_ctx.h"

void cm_ctx_release_extras(cm_ctx *c) { (void)c; }
