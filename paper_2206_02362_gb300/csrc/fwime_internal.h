// Internal links between the translation units of libfwime (not part of the C ABI).
#pragma once
#include "../../include/fwime.h"

namespace fwk {

struct Server;                                   // the request server (fwime_serve.cu)

// A context that carries a server instead of a grid (fwime_server_create); operator calls on it fail.
fwime_ctx *ctx_for_server(Server *srv);
Server *ctx_server(const fwime_ctx *x);
// Stops the server's threads after every submitted request has finished, and frees it.
void server_destroy(Server *srv);
// Waits until every request submitted so far has finished (fwime_sync on a server context).
int server_sync(Server *srv);

}  // namespace fwk
