// ws_inst_u8_shapes.cu -- instantiates the 2D pipelines for 8-bit gradients on
// the tile shapes other than the default one (ws_tuning.tile_shape 1..3; the
// template value is CONN + 100 * shape).
#include "ws_launch.cuh"

namespace ws {

const Launchers *launchers_u8_shape(int conn, int shape)
{
    switch (conn + 100 * shape) {
    case 104: return Inst<uint8_t, 104>::get();
    case 108: return Inst<uint8_t, 108>::get();
    case 204: return Inst<uint8_t, 204>::get();
    case 208: return Inst<uint8_t, 208>::get();
    case 304: return Inst<uint8_t, 304>::get();
    case 308: return Inst<uint8_t, 308>::get();
    default: return nullptr;
    }
}

}  // namespace ws
