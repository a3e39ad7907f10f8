"""The device's default memory pool (where cudaMallocAsync draws from), read
through the CUDA driver API: used by the tests that show a call allocates
nothing."""
import ctypes

# CUmemPool_attribute values of the CUDA driver API (cuda.h)
RESERVED_MEM_CURRENT, USED_MEM_CURRENT, USED_MEM_HIGH = 5, 7, 8


class Pool:
    def __init__(self, ordinal):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)  # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def snapshot(self):
        """Pool reserved and used bytes, torch's allocated and reserved bytes,
        the device's free memory."""
        import torch
        return (self.get(RESERVED_MEM_CURRENT), self.get(USED_MEM_CURRENT),
                torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
                torch.cuda.mem_get_info()[0])
