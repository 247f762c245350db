// kf_device.h -- the current-device guard of every entry point (library-internal).
#pragma once

#include <cuda_runtime.h>

namespace kf {

// Makes `device` current for the scope of one library call and makes the caller's
// current device current again when the scope ends, so a host thread that drives
// several GPUs through several contexts keeps the device it chose. Nothing is switched
// (and nothing restored) when the caller's device already is `device`.
class DeviceScope {
public:
    explicit DeviceScope(int device)
    {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        err_ = (prev_ == device) ? cudaSuccess : cudaSetDevice(device);
        switched_ = err_ == cudaSuccess && prev_ >= 0 && prev_ != device;
    }
    ~DeviceScope()
    {
        if (switched_) cudaSetDevice(prev_);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
    cudaError_t status() const { return err_; }

private:
    int prev_ = -1;
    bool switched_ = false;
    cudaError_t err_ = cudaSuccess;
};

}  // namespace kf
