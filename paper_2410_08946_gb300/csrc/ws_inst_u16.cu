// ws_inst_u16.cu -- instantiates the pipelines for 16-bit gradients.
#include "ws_launch.cuh"

namespace ws {

const Launchers *launchers_u16(int conn)
{
    switch (conn) {
    case 4: return Inst<uint16_t, 4>::get();
    case 8: return Inst<uint16_t, 8>::get();
    case 6: return Inst<uint16_t, 6>::get();
    case 26: return Inst<uint16_t, 26>::get();
    default: return nullptr;
    }
}

}  // namespace ws
