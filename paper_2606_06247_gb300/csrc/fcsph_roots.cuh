// Generated by gen_roots.py: cos and sin of 2 pi e / N for the composite
// register-DFT sizes N.  Do not edit by hand.
#pragma once

namespace fcsph {

template <int N> __device__ __forceinline__ float rcos(int e);
template <int N> __device__ __forceinline__ float rsin(int e);

template <> __device__ __forceinline__ float rcos<6>(int e) {
  switch (((e % 6) + 6) % 6) {
    case 0: return 1.0f;
    case 1: return 0.5f;
    case 2: return -0.5f;
    case 3: return -1.0f;
    case 4: return -0.5f;
    case 5: return 0.5f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<6>(int e) {
  switch (((e % 6) + 6) % 6) {
    case 0: return 0.0f;
    case 1: return 0.86602540378443865f;
    case 2: return 0.86602540378443865f;
    case 3: return 4.1340642196527976e-43f;
    case 4: return -0.86602540378443865f;
    case 5: return -0.86602540378443865f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<10>(int e) {
  switch (((e % 10) + 10) % 10) {
    case 0: return 1.0f;
    case 1: return 0.80901699437494742f;
    case 2: return 0.30901699437494742f;
    case 3: return -0.30901699437494742f;
    case 4: return -0.80901699437494742f;
    case 5: return -1.0f;
    case 6: return -0.80901699437494742f;
    case 7: return -0.30901699437494742f;
    case 8: return 0.30901699437494742f;
    case 9: return 0.80901699437494742f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<10>(int e) {
  switch (((e % 10) + 10) % 10) {
    case 0: return 0.0f;
    case 1: return 0.58778525229247313f;
    case 2: return 0.95105651629515357f;
    case 3: return 0.95105651629515357f;
    case 4: return 0.58778525229247313f;
    case 5: return 4.1340642196527976e-43f;
    case 6: return -0.58778525229247313f;
    case 7: return -0.95105651629515357f;
    case 8: return -0.95105651629515357f;
    case 9: return -0.58778525229247313f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<14>(int e) {
  switch (((e % 14) + 14) % 14) {
    case 0: return 1.0f;
    case 1: return 0.90096886790241913f;
    case 2: return 0.62348980185873353f;
    case 3: return 0.2225209339563144f;
    case 4: return -0.2225209339563144f;
    case 5: return -0.62348980185873353f;
    case 6: return -0.90096886790241913f;
    case 7: return -1.0f;
    case 8: return -0.90096886790241913f;
    case 9: return -0.62348980185873353f;
    case 10: return -0.2225209339563144f;
    case 11: return 0.2225209339563144f;
    case 12: return 0.62348980185873353f;
    case 13: return 0.90096886790241913f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<14>(int e) {
  switch (((e % 14) + 14) % 14) {
    case 0: return 0.0f;
    case 1: return 0.43388373911755812f;
    case 2: return 0.78183148246802981f;
    case 3: return 0.97492791218182361f;
    case 4: return 0.97492791218182361f;
    case 5: return 0.78183148246802981f;
    case 6: return 0.43388373911755812f;
    case 7: return 4.1340642196527976e-43f;
    case 8: return -0.43388373911755812f;
    case 9: return -0.78183148246802981f;
    case 10: return -0.97492791218182361f;
    case 11: return -0.97492791218182361f;
    case 12: return -0.78183148246802981f;
    case 13: return -0.43388373911755812f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<15>(int e) {
  switch (((e % 15) + 15) % 15) {
    case 0: return 1.0f;
    case 1: return 0.9135454576426009f;
    case 2: return 0.66913060635885821f;
    case 3: return 0.30901699437494742f;
    case 4: return -0.10452846326765347f;
    case 5: return -0.5f;
    case 6: return -0.80901699437494742f;
    case 7: return -0.97814760073380564f;
    case 8: return -0.97814760073380564f;
    case 9: return -0.80901699437494742f;
    case 10: return -0.5f;
    case 11: return -0.10452846326765347f;
    case 12: return 0.30901699437494742f;
    case 13: return 0.66913060635885821f;
    case 14: return 0.9135454576426009f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<15>(int e) {
  switch (((e % 15) + 15) % 15) {
    case 0: return 0.0f;
    case 1: return 0.40673664307580021f;
    case 2: return 0.74314482547739424f;
    case 3: return 0.95105651629515357f;
    case 4: return 0.99452189536827334f;
    case 5: return 0.86602540378443865f;
    case 6: return 0.58778525229247313f;
    case 7: return 0.20791169081775934f;
    case 8: return -0.20791169081775934f;
    case 9: return -0.58778525229247313f;
    case 10: return -0.86602540378443865f;
    case 11: return -0.99452189536827334f;
    case 12: return -0.95105651629515357f;
    case 13: return -0.74314482547739424f;
    case 14: return -0.40673664307580021f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<20>(int e) {
  switch (((e % 20) + 20) % 20) {
    case 0: return 1.0f;
    case 1: return 0.95105651629515357f;
    case 2: return 0.80901699437494742f;
    case 3: return 0.58778525229247313f;
    case 4: return 0.30901699437494742f;
    case 5: return 2.0670321098263988e-43f;
    case 6: return -0.30901699437494742f;
    case 7: return -0.58778525229247313f;
    case 8: return -0.80901699437494742f;
    case 9: return -0.95105651629515357f;
    case 10: return -1.0f;
    case 11: return -0.95105651629515357f;
    case 12: return -0.80901699437494742f;
    case 13: return -0.58778525229247313f;
    case 14: return -0.30901699437494742f;
    case 15: return -6.9496731751441328e-41f;
    case 16: return 0.30901699437494742f;
    case 17: return 0.58778525229247313f;
    case 18: return 0.80901699437494742f;
    case 19: return 0.95105651629515357f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<20>(int e) {
  switch (((e % 20) + 20) % 20) {
    case 0: return 0.0f;
    case 1: return 0.30901699437494742f;
    case 2: return 0.58778525229247313f;
    case 3: return 0.80901699437494742f;
    case 4: return 0.95105651629515357f;
    case 5: return 1.0f;
    case 6: return 0.95105651629515357f;
    case 7: return 0.80901699437494742f;
    case 8: return 0.58778525229247313f;
    case 9: return 0.30901699437494742f;
    case 10: return 4.1340642196527976e-43f;
    case 11: return -0.30901699437494742f;
    case 12: return -0.58778525229247313f;
    case 13: return -0.80901699437494742f;
    case 14: return -0.95105651629515357f;
    case 15: return -1.0f;
    case 16: return -0.95105651629515357f;
    case 17: return -0.80901699437494742f;
    case 18: return -0.58778525229247313f;
    case 19: return -0.30901699437494742f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<21>(int e) {
  switch (((e % 21) + 21) % 21) {
    case 0: return 1.0f;
    case 1: return 0.95557280578614073f;
    case 2: return 0.82623877431599487f;
    case 3: return 0.62348980185873353f;
    case 4: return 0.36534102436639501f;
    case 5: return 7.4730093586424254e-2f;
    case 6: return -0.2225209339563144f;
    case 7: return -0.5f;
    case 8: return -0.73305187182982633f;
    case 9: return -0.90096886790241913f;
    case 10: return -0.98883082622512855f;
    case 11: return -0.98883082622512855f;
    case 12: return -0.90096886790241913f;
    case 13: return -0.73305187182982633f;
    case 14: return -0.5f;
    case 15: return -0.2225209339563144f;
    case 16: return 7.4730093586424254e-2f;
    case 17: return 0.36534102436639501f;
    case 18: return 0.62348980185873353f;
    case 19: return 0.82623877431599487f;
    case 20: return 0.95557280578614073f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<21>(int e) {
  switch (((e % 21) + 21) % 21) {
    case 0: return 0.0f;
    case 1: return 0.29475517441090422f;
    case 2: return 0.56332005806362203f;
    case 3: return 0.78183148246802981f;
    case 4: return 0.93087374864420426f;
    case 5: return 0.99720379718118015f;
    case 6: return 0.97492791218182361f;
    case 7: return 0.86602540378443865f;
    case 8: return 0.68017273777091939f;
    case 9: return 0.43388373911755812f;
    case 10: return 0.14904226617617445f;
    case 11: return -0.14904226617617445f;
    case 12: return -0.43388373911755812f;
    case 13: return -0.68017273777091939f;
    case 14: return -0.86602540378443865f;
    case 15: return -0.97492791218182361f;
    case 16: return -0.99720379718118015f;
    case 17: return -0.93087374864420426f;
    case 18: return -0.78183148246802981f;
    case 19: return -0.56332005806362203f;
    case 20: return -0.29475517441090422f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<25>(int e) {
  switch (((e % 25) + 25) % 25) {
    case 0: return 1.0f;
    case 1: return 0.96858316112863112f;
    case 2: return 0.87630668004386359f;
    case 3: return 0.72896862742141152f;
    case 4: return 0.53582679497899662f;
    case 5: return 0.30901699437494742f;
    case 6: return 6.2790519529313376e-2f;
    case 7: return -0.18738131458572463f;
    case 8: return -0.42577929156507265f;
    case 9: return -0.63742398974868971f;
    case 10: return -0.80901699437494742f;
    case 11: return -0.9297764858882514f;
    case 12: return -0.99211470131447783f;
    case 13: return -0.99211470131447783f;
    case 14: return -0.9297764858882514f;
    case 15: return -0.80901699437494742f;
    case 16: return -0.63742398974868971f;
    case 17: return -0.42577929156507265f;
    case 18: return -0.18738131458572463f;
    case 19: return 6.2790519529313376e-2f;
    case 20: return 0.30901699437494742f;
    case 21: return 0.53582679497899662f;
    case 22: return 0.72896862742141152f;
    case 23: return 0.87630668004386359f;
    case 24: return 0.96858316112863112f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<25>(int e) {
  switch (((e % 25) + 25) % 25) {
    case 0: return 0.0f;
    case 1: return 0.24868988716485479f;
    case 2: return 0.48175367410171527f;
    case 3: return 0.68454710592868867f;
    case 4: return 0.84432792550201508f;
    case 5: return 0.95105651629515357f;
    case 6: return 0.99802672842827156f;
    case 7: return 0.98228725072868868f;
    case 8: return 0.90482705246601953f;
    case 9: return 0.77051324277578923f;
    case 10: return 0.58778525229247313f;
    case 11: return 0.36812455268467796f;
    case 12: return 0.12533323356430425f;
    case 13: return -0.12533323356430425f;
    case 14: return -0.36812455268467796f;
    case 15: return -0.58778525229247313f;
    case 16: return -0.77051324277578923f;
    case 17: return -0.90482705246601953f;
    case 18: return -0.98228725072868868f;
    case 19: return -0.99802672842827156f;
    case 20: return -0.95105651629515357f;
    case 21: return -0.84432792550201508f;
    case 22: return -0.68454710592868867f;
    case 23: return -0.48175367410171527f;
    case 24: return -0.24868988716485479f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<27>(int e) {
  switch (((e % 27) + 27) % 27) {
    case 0: return 1.0f;
    case 1: return 0.97304487057982384f;
    case 2: return 0.89363264032341225f;
    case 3: return 0.76604444311897804f;
    case 4: return 0.59715859170278616f;
    case 5: return 0.39607976603915682f;
    case 6: return 0.17364817766693035f;
    case 7: return -5.8144828910475829e-2f;
    case 8: return -0.28680323271109025f;
    case 9: return -0.5f;
    case 10: return -0.68624163786873359f;
    case 11: return -0.83548781141293642f;
    case 12: return -0.93969262078590838f;
    case 13: return -0.99323835774194299f;
    case 14: return -0.99323835774194299f;
    case 15: return -0.93969262078590838f;
    case 16: return -0.83548781141293642f;
    case 17: return -0.68624163786873359f;
    case 18: return -0.5f;
    case 19: return -0.28680323271109025f;
    case 20: return -5.8144828910475829e-2f;
    case 21: return 0.17364817766693035f;
    case 22: return 0.39607976603915682f;
    case 23: return 0.59715859170278616f;
    case 24: return 0.76604444311897804f;
    case 25: return 0.89363264032341225f;
    case 26: return 0.97304487057982384f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<27>(int e) {
  switch (((e % 27) + 27) % 27) {
    case 0: return 0.0f;
    case 1: return 0.23061587074244018f;
    case 2: return 0.44879918020046217f;
    case 3: return 0.64278760968653933f;
    case 4: return 0.80212319275504379f;
    case 5: return 0.91821610688027401f;
    case 6: return 0.98480775301220806f;
    case 7: return 0.99830815827126821f;
    case 8: return 0.95798951231548887f;
    case 9: return 0.86602540378443865f;
    case 10: return 0.7273736415730487f;
    case 11: return 0.54950897807080604f;
    case 12: return 0.34202014332566873f;
    case 13: return 0.11609291412523023f;
    case 14: return -0.11609291412523023f;
    case 15: return -0.34202014332566873f;
    case 16: return -0.54950897807080604f;
    case 17: return -0.7273736415730487f;
    case 18: return -0.86602540378443865f;
    case 19: return -0.95798951231548887f;
    case 20: return -0.99830815827126821f;
    case 21: return -0.98480775301220806f;
    case 22: return -0.91821610688027401f;
    case 23: return -0.80212319275504379f;
    case 24: return -0.64278760968653933f;
    case 25: return -0.44879918020046217f;
    case 26: return -0.23061587074244018f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<28>(int e) {
  switch (((e % 28) + 28) % 28) {
    case 0: return 1.0f;
    case 1: return 0.97492791218182361f;
    case 2: return 0.90096886790241913f;
    case 3: return 0.78183148246802981f;
    case 4: return 0.62348980185873353f;
    case 5: return 0.43388373911755812f;
    case 6: return 0.2225209339563144f;
    case 7: return 2.0670321098263988e-43f;
    case 8: return -0.2225209339563144f;
    case 9: return -0.43388373911755812f;
    case 10: return -0.62348980185873353f;
    case 11: return -0.78183148246802981f;
    case 12: return -0.90096886790241913f;
    case 13: return -0.97492791218182361f;
    case 14: return -1.0f;
    case 15: return -0.97492791218182361f;
    case 16: return -0.90096886790241913f;
    case 17: return -0.78183148246802981f;
    case 18: return -0.62348980185873353f;
    case 19: return -0.43388373911755812f;
    case 20: return -0.2225209339563144f;
    case 21: return 2.2338764406549883e-41f;
    case 22: return 0.2225209339563144f;
    case 23: return 0.43388373911755812f;
    case 24: return 0.62348980185873353f;
    case 25: return 0.78183148246802981f;
    case 26: return 0.90096886790241913f;
    case 27: return 0.97492791218182361f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<28>(int e) {
  switch (((e % 28) + 28) % 28) {
    case 0: return 0.0f;
    case 1: return 0.2225209339563144f;
    case 2: return 0.43388373911755812f;
    case 3: return 0.62348980185873353f;
    case 4: return 0.78183148246802981f;
    case 5: return 0.90096886790241913f;
    case 6: return 0.97492791218182361f;
    case 7: return 1.0f;
    case 8: return 0.97492791218182361f;
    case 9: return 0.90096886790241913f;
    case 10: return 0.78183148246802981f;
    case 11: return 0.62348980185873353f;
    case 12: return 0.43388373911755812f;
    case 13: return 0.2225209339563144f;
    case 14: return 4.1340642196527976e-43f;
    case 15: return -0.2225209339563144f;
    case 16: return -0.43388373911755812f;
    case 17: return -0.62348980185873353f;
    case 18: return -0.78183148246802981f;
    case 19: return -0.90096886790241913f;
    case 20: return -0.97492791218182361f;
    case 21: return -1.0f;
    case 22: return -0.97492791218182361f;
    case 23: return -0.90096886790241913f;
    case 24: return -0.78183148246802981f;
    case 25: return -0.62348980185873353f;
    case 26: return -0.43388373911755812f;
    case 27: return -0.2225209339563144f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<30>(int e) {
  switch (((e % 30) + 30) % 30) {
    case 0: return 1.0f;
    case 1: return 0.97814760073380564f;
    case 2: return 0.9135454576426009f;
    case 3: return 0.80901699437494742f;
    case 4: return 0.66913060635885821f;
    case 5: return 0.5f;
    case 6: return 0.30901699437494742f;
    case 7: return 0.10452846326765347f;
    case 8: return -0.10452846326765347f;
    case 9: return -0.30901699437494742f;
    case 10: return -0.5f;
    case 11: return -0.66913060635885821f;
    case 12: return -0.80901699437494742f;
    case 13: return -0.9135454576426009f;
    case 14: return -0.97814760073380564f;
    case 15: return -1.0f;
    case 16: return -0.97814760073380564f;
    case 17: return -0.9135454576426009f;
    case 18: return -0.80901699437494742f;
    case 19: return -0.66913060635885821f;
    case 20: return -0.5f;
    case 21: return -0.30901699437494742f;
    case 22: return -0.10452846326765347f;
    case 23: return 0.10452846326765347f;
    case 24: return 0.30901699437494742f;
    case 25: return 0.5f;
    case 26: return 0.66913060635885821f;
    case 27: return 0.80901699437494742f;
    case 28: return 0.9135454576426009f;
    case 29: return 0.97814760073380564f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<30>(int e) {
  switch (((e % 30) + 30) % 30) {
    case 0: return 0.0f;
    case 1: return 0.20791169081775934f;
    case 2: return 0.40673664307580021f;
    case 3: return 0.58778525229247313f;
    case 4: return 0.74314482547739424f;
    case 5: return 0.86602540378443865f;
    case 6: return 0.95105651629515357f;
    case 7: return 0.99452189536827334f;
    case 8: return 0.99452189536827334f;
    case 9: return 0.95105651629515357f;
    case 10: return 0.86602540378443865f;
    case 11: return 0.74314482547739424f;
    case 12: return 0.58778525229247313f;
    case 13: return 0.40673664307580021f;
    case 14: return 0.20791169081775934f;
    case 15: return 4.1340642196527976e-43f;
    case 16: return -0.20791169081775934f;
    case 17: return -0.40673664307580021f;
    case 18: return -0.58778525229247313f;
    case 19: return -0.74314482547739424f;
    case 20: return -0.86602540378443865f;
    case 21: return -0.95105651629515357f;
    case 22: return -0.99452189536827334f;
    case 23: return -0.99452189536827334f;
    case 24: return -0.95105651629515357f;
    case 25: return -0.86602540378443865f;
    case 26: return -0.74314482547739424f;
    case 27: return -0.58778525229247313f;
    case 28: return -0.40673664307580021f;
    case 29: return -0.20791169081775934f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<35>(int e) {
  switch (((e % 35) + 35) % 35) {
    case 0: return 1.0f;
    case 1: return 0.98392958859862966f;
    case 2: return 0.93623487063973721f;
    case 3: return 0.85844879360186612f;
    case 4: return 0.75307146600361093f;
    case 5: return 0.62348980185873353f;
    case 6: return 0.47386866247299867f;
    case 7: return 0.30901699437494742f;
    case 8: return 0.13423326581765548f;
    case 9: return -4.4864830350514925e-2f;
    case 10: return -0.2225209339563144f;
    case 11: return -0.39302503165392362f;
    case 12: return -0.55089698145210252f;
    case 13: return -0.69106264898686468f;
    case 14: return -0.80901699437494742f;
    case 15: return -0.90096886790241913f;
    case 16: return -0.96396286069585329f;
    case 17: return -0.99597429399523903f;
    case 18: return -0.99597429399523903f;
    case 19: return -0.96396286069585329f;
    case 20: return -0.90096886790241913f;
    case 21: return -0.80901699437494742f;
    case 22: return -0.69106264898686468f;
    case 23: return -0.55089698145210252f;
    case 24: return -0.39302503165392362f;
    case 25: return -0.2225209339563144f;
    case 26: return -4.4864830350514925e-2f;
    case 27: return 0.13423326581765548f;
    case 28: return 0.30901699437494742f;
    case 29: return 0.47386866247299867f;
    case 30: return 0.62348980185873353f;
    case 31: return 0.75307146600361093f;
    case 32: return 0.85844879360186612f;
    case 33: return 0.93623487063973721f;
    case 34: return 0.98392958859862966f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<35>(int e) {
  switch (((e % 35) + 35) % 35) {
    case 0: return 0.0f;
    case 1: return 0.17855689479863665f;
    case 2: return 0.3513748240813427f;
    case 3: return 0.51289927740590614f;
    case 4: return 0.65793872593971261f;
    case 5: return 0.78183148246802981f;
    case 6: return 0.880595531856738f;
    case 7: return 0.95105651629515357f;
    case 8: return 0.99094976176793476f;
    case 9: return 0.99899306654131465f;
    case 10: return 0.97492791218182361f;
    case 11: return 0.91952777255145064f;
    case 12: return 0.83457325372130265f;
    case 13: return 0.72279486382739153f;
    case 14: return 0.58778525229247313f;
    case 15: return 0.43388373911755812f;
    case 16: return 0.26603684556667511f;
    case 17: return 8.96393089034335e-2f;
    case 18: return -8.96393089034335e-2f;
    case 19: return -0.26603684556667511f;
    case 20: return -0.43388373911755812f;
    case 21: return -0.58778525229247313f;
    case 22: return -0.72279486382739153f;
    case 23: return -0.83457325372130265f;
    case 24: return -0.91952777255145064f;
    case 25: return -0.97492791218182361f;
    case 26: return -0.99899306654131465f;
    case 27: return -0.99094976176793476f;
    case 28: return -0.95105651629515357f;
    case 29: return -0.880595531856738f;
    case 30: return -0.78183148246802981f;
    case 31: return -0.65793872593971261f;
    case 32: return -0.51289927740590614f;
    case 33: return -0.3513748240813427f;
    case 34: return -0.17855689479863665f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<36>(int e) {
  switch (((e % 36) + 36) % 36) {
    case 0: return 1.0f;
    case 1: return 0.98480775301220806f;
    case 2: return 0.93969262078590838f;
    case 3: return 0.86602540378443865f;
    case 4: return 0.76604444311897804f;
    case 5: return 0.64278760968653933f;
    case 6: return 0.5f;
    case 7: return 0.34202014332566873f;
    case 8: return 0.17364817766693035f;
    case 9: return 2.0670321098263988e-43f;
    case 10: return -0.17364817766693035f;
    case 11: return -0.34202014332566873f;
    case 12: return -0.5f;
    case 13: return -0.64278760968653933f;
    case 14: return -0.76604444311897804f;
    case 15: return -0.86602540378443865f;
    case 16: return -0.93969262078590838f;
    case 17: return -0.98480775301220806f;
    case 18: return -1.0f;
    case 19: return -0.98480775301220806f;
    case 20: return -0.93969262078590838f;
    case 21: return -0.86602540378443865f;
    case 22: return -0.76604444311897804f;
    case 23: return -0.64278760968653933f;
    case 24: return -0.5f;
    case 25: return -0.34202014332566873f;
    case 26: return -0.17364817766693035f;
    case 27: return 2.2338764406549883e-41f;
    case 28: return 0.17364817766693035f;
    case 29: return 0.34202014332566873f;
    case 30: return 0.5f;
    case 31: return 0.64278760968653933f;
    case 32: return 0.76604444311897804f;
    case 33: return 0.86602540378443865f;
    case 34: return 0.93969262078590838f;
    case 35: return 0.98480775301220806f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<36>(int e) {
  switch (((e % 36) + 36) % 36) {
    case 0: return 0.0f;
    case 1: return 0.17364817766693035f;
    case 2: return 0.34202014332566873f;
    case 3: return 0.5f;
    case 4: return 0.64278760968653933f;
    case 5: return 0.76604444311897804f;
    case 6: return 0.86602540378443865f;
    case 7: return 0.93969262078590838f;
    case 8: return 0.98480775301220806f;
    case 9: return 1.0f;
    case 10: return 0.98480775301220806f;
    case 11: return 0.93969262078590838f;
    case 12: return 0.86602540378443865f;
    case 13: return 0.76604444311897804f;
    case 14: return 0.64278760968653933f;
    case 15: return 0.5f;
    case 16: return 0.34202014332566873f;
    case 17: return 0.17364817766693035f;
    case 18: return 4.1340642196527976e-43f;
    case 19: return -0.17364817766693035f;
    case 20: return -0.34202014332566873f;
    case 21: return -0.5f;
    case 22: return -0.64278760968653933f;
    case 23: return -0.76604444311897804f;
    case 24: return -0.86602540378443865f;
    case 25: return -0.93969262078590838f;
    case 26: return -0.98480775301220806f;
    case 27: return -1.0f;
    case 28: return -0.98480775301220806f;
    case 29: return -0.93969262078590838f;
    case 30: return -0.86602540378443865f;
    case 31: return -0.76604444311897804f;
    case 32: return -0.64278760968653933f;
    case 33: return -0.5f;
    case 34: return -0.34202014332566873f;
    case 35: return -0.17364817766693035f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<42>(int e) {
  switch (((e % 42) + 42) % 42) {
    case 0: return 1.0f;
    case 1: return 0.98883082622512855f;
    case 2: return 0.95557280578614073f;
    case 3: return 0.90096886790241913f;
    case 4: return 0.82623877431599487f;
    case 5: return 0.73305187182982633f;
    case 6: return 0.62348980185873353f;
    case 7: return 0.5f;
    case 8: return 0.36534102436639501f;
    case 9: return 0.2225209339563144f;
    case 10: return 7.4730093586424254e-2f;
    case 11: return -7.4730093586424254e-2f;
    case 12: return -0.2225209339563144f;
    case 13: return -0.36534102436639501f;
    case 14: return -0.5f;
    case 15: return -0.62348980185873353f;
    case 16: return -0.73305187182982633f;
    case 17: return -0.82623877431599487f;
    case 18: return -0.90096886790241913f;
    case 19: return -0.95557280578614073f;
    case 20: return -0.98883082622512855f;
    case 21: return -1.0f;
    case 22: return -0.98883082622512855f;
    case 23: return -0.95557280578614073f;
    case 24: return -0.90096886790241913f;
    case 25: return -0.82623877431599487f;
    case 26: return -0.73305187182982633f;
    case 27: return -0.62348980185873353f;
    case 28: return -0.5f;
    case 29: return -0.36534102436639501f;
    case 30: return -0.2225209339563144f;
    case 31: return -7.4730093586424254e-2f;
    case 32: return 7.4730093586424254e-2f;
    case 33: return 0.2225209339563144f;
    case 34: return 0.36534102436639501f;
    case 35: return 0.5f;
    case 36: return 0.62348980185873353f;
    case 37: return 0.73305187182982633f;
    case 38: return 0.82623877431599487f;
    case 39: return 0.90096886790241913f;
    case 40: return 0.95557280578614073f;
    case 41: return 0.98883082622512855f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<42>(int e) {
  switch (((e % 42) + 42) % 42) {
    case 0: return 0.0f;
    case 1: return 0.14904226617617445f;
    case 2: return 0.29475517441090422f;
    case 3: return 0.43388373911755812f;
    case 4: return 0.56332005806362203f;
    case 5: return 0.68017273777091939f;
    case 6: return 0.78183148246802981f;
    case 7: return 0.86602540378443865f;
    case 8: return 0.93087374864420426f;
    case 9: return 0.97492791218182361f;
    case 10: return 0.99720379718118015f;
    case 11: return 0.99720379718118015f;
    case 12: return 0.97492791218182361f;
    case 13: return 0.93087374864420426f;
    case 14: return 0.86602540378443865f;
    case 15: return 0.78183148246802981f;
    case 16: return 0.68017273777091939f;
    case 17: return 0.56332005806362203f;
    case 18: return 0.43388373911755812f;
    case 19: return 0.29475517441090422f;
    case 20: return 0.14904226617617445f;
    case 21: return 4.1340642196527976e-43f;
    case 22: return -0.14904226617617445f;
    case 23: return -0.29475517441090422f;
    case 24: return -0.43388373911755812f;
    case 25: return -0.56332005806362203f;
    case 26: return -0.68017273777091939f;
    case 27: return -0.78183148246802981f;
    case 28: return -0.86602540378443865f;
    case 29: return -0.93087374864420426f;
    case 30: return -0.97492791218182361f;
    case 31: return -0.99720379718118015f;
    case 32: return -0.99720379718118015f;
    case 33: return -0.97492791218182361f;
    case 34: return -0.93087374864420426f;
    case 35: return -0.86602540378443865f;
    case 36: return -0.78183148246802981f;
    case 37: return -0.68017273777091939f;
    case 38: return -0.56332005806362203f;
    case 39: return -0.43388373911755812f;
    case 40: return -0.29475517441090422f;
    case 41: return -0.14904226617617445f;
    default: return 0.0f;
  }
}

template <> __device__ __forceinline__ float rcos<50>(int e) {
  switch (((e % 50) + 50) % 50) {
    case 0: return 1.0f;
    case 1: return 0.99211470131447783f;
    case 2: return 0.96858316112863112f;
    case 3: return 0.9297764858882514f;
    case 4: return 0.87630668004386359f;
    case 5: return 0.80901699437494742f;
    case 6: return 0.72896862742141152f;
    case 7: return 0.63742398974868971f;
    case 8: return 0.53582679497899662f;
    case 9: return 0.42577929156507265f;
    case 10: return 0.30901699437494742f;
    case 11: return 0.18738131458572463f;
    case 12: return 6.2790519529313376e-2f;
    case 13: return -6.2790519529313376e-2f;
    case 14: return -0.18738131458572463f;
    case 15: return -0.30901699437494742f;
    case 16: return -0.42577929156507265f;
    case 17: return -0.53582679497899662f;
    case 18: return -0.63742398974868971f;
    case 19: return -0.72896862742141152f;
    case 20: return -0.80901699437494742f;
    case 21: return -0.87630668004386359f;
    case 22: return -0.9297764858882514f;
    case 23: return -0.96858316112863112f;
    case 24: return -0.99211470131447783f;
    case 25: return -1.0f;
    case 26: return -0.99211470131447783f;
    case 27: return -0.96858316112863112f;
    case 28: return -0.9297764858882514f;
    case 29: return -0.87630668004386359f;
    case 30: return -0.80901699437494742f;
    case 31: return -0.72896862742141152f;
    case 32: return -0.63742398974868971f;
    case 33: return -0.53582679497899662f;
    case 34: return -0.42577929156507265f;
    case 35: return -0.30901699437494742f;
    case 36: return -0.18738131458572463f;
    case 37: return -6.2790519529313376e-2f;
    case 38: return 6.2790519529313376e-2f;
    case 39: return 0.18738131458572463f;
    case 40: return 0.30901699437494742f;
    case 41: return 0.42577929156507265f;
    case 42: return 0.53582679497899662f;
    case 43: return 0.63742398974868971f;
    case 44: return 0.72896862742141152f;
    case 45: return 0.80901699437494742f;
    case 46: return 0.87630668004386359f;
    case 47: return 0.9297764858882514f;
    case 48: return 0.96858316112863112f;
    case 49: return 0.99211470131447783f;
    default: return 0.0f;
  }
}
template <> __device__ __forceinline__ float rsin<50>(int e) {
  switch (((e % 50) + 50) % 50) {
    case 0: return 0.0f;
    case 1: return 0.12533323356430425f;
    case 2: return 0.24868988716485479f;
    case 3: return 0.36812455268467796f;
    case 4: return 0.48175367410171527f;
    case 5: return 0.58778525229247313f;
    case 6: return 0.68454710592868867f;
    case 7: return 0.77051324277578923f;
    case 8: return 0.84432792550201508f;
    case 9: return 0.90482705246601953f;
    case 10: return 0.95105651629515357f;
    case 11: return 0.98228725072868868f;
    case 12: return 0.99802672842827156f;
    case 13: return 0.99802672842827156f;
    case 14: return 0.98228725072868868f;
    case 15: return 0.95105651629515357f;
    case 16: return 0.90482705246601953f;
    case 17: return 0.84432792550201508f;
    case 18: return 0.77051324277578923f;
    case 19: return 0.68454710592868867f;
    case 20: return 0.58778525229247313f;
    case 21: return 0.48175367410171527f;
    case 22: return 0.36812455268467796f;
    case 23: return 0.24868988716485479f;
    case 24: return 0.12533323356430425f;
    case 25: return 4.1340642196527976e-43f;
    case 26: return -0.12533323356430425f;
    case 27: return -0.24868988716485479f;
    case 28: return -0.36812455268467796f;
    case 29: return -0.48175367410171527f;
    case 30: return -0.58778525229247313f;
    case 31: return -0.68454710592868867f;
    case 32: return -0.77051324277578923f;
    case 33: return -0.84432792550201508f;
    case 34: return -0.90482705246601953f;
    case 35: return -0.95105651629515357f;
    case 36: return -0.98228725072868868f;
    case 37: return -0.99802672842827156f;
    case 38: return -0.99802672842827156f;
    case 39: return -0.98228725072868868f;
    case 40: return -0.95105651629515357f;
    case 41: return -0.90482705246601953f;
    case 42: return -0.84432792550201508f;
    case 43: return -0.77051324277578923f;
    case 44: return -0.68454710592868867f;
    case 45: return -0.58778525229247313f;
    case 46: return -0.48175367410171527f;
    case 47: return -0.36812455268467796f;
    case 48: return -0.24868988716485479f;
    case 49: return -0.12533323356430425f;
    default: return 0.0f;
  }
}

}  // namespace fcsph
