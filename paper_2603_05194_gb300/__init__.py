"""GB300-native PCG-ATKM ground-state solver for rotating dipolar BECs.

The compute path is the C-ABI CUDA library ``libatkm.so`` (include/atkm.h),
built in-tree for sm_103a by ``paper_2603_05194_gb300.build``; the Python
binding in ``binding`` only marshals tensors into it.
"""
