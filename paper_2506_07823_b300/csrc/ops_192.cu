// ops_192.cu -- kernel instantiations of one size class.
#include "ops_impl.cuh"

namespace pdl {

const SizeOps* ops_192(int n, int m)
{
    static const SizeOps table[] = {make_ops<192, 192, true, true>()};
    for (const auto& o : table)
        if (o.n == n && o.m == m) return &o;
    return nullptr;
}

}  // namespace pdl
