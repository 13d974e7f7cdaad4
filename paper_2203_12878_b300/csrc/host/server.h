// Continuous-batching check server (see drf_server_* in include/drf.h).
#pragma once

struct drf_ctx;

namespace drf {
class Server;
}
