"""GB300-native ChiSao population step (sm_103a CUDA behind a C ABI).

``chisao`` holds the ctypes binding of the C ABI declared in include/chisao.h;
``inputs`` the seeded synthetic workloads.
"""
