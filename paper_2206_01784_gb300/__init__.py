"""GB300-native Onesweep LSD radix sort (Adinets and Merrill, arXiv 2206.01784).

The sort runs in hand-written CUDA kernels for sm_103a behind a C ABI
(``include/onesweep.h``, built into ``libonesweep.so``). ``onesweep`` is the
thin Python binding; ``workload`` draws the seeded synthetic inputs.
"""
